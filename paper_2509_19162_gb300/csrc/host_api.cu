// Host driver and C ABI of the growth library (declarations and contracts in
// include/cg_growth.h).
//
// A growth job (Section 2.1, Def. "Growth") is run by the hash strategy: one persistent,
// cooperative kernel launch performs every layer step (hash_path.cu).  The host only plans
// device memory, uploads the job, and reads the layer sizes back.  When a layer outgrows the
// job's buffers the kernel stops at the last complete layer; the host then grows the buffers
// (within mem_cap), rebuilds the visited table from the stored states and relaunches.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "../../include/cg_growth.h"
#include "cg_device.cuh"
#include "cg_internal.h"
#include "cg_kernels.h"
#include "group_order.h"
#include "sort_kernels.h"

using cg::Ctl;
using cg::GenSM;
using cg::JobDev;
using cg::SweepDev;

namespace {

constexpr uint64_t kDefaultMemCap = 160ull << 30;
constexpr uint64_t kTimeoutNs = 30ull * 1000 * 1000 * 1000;  // per barrier wait
// A sweep round of all of S_14 can take seconds; a block with no work waits that long.
constexpr uint64_t kSweepTimeoutNs = 120ull * 1000 * 1000 * 1000;
// A growth whose rank bitmap exceeds L2 orders frontiers of at least this many states by rank
// before expanding them (run_hash); smaller ones cost more to order than the L2 hits buy.
constexpr uint64_t kOrderMinStates = 1ull << 20;
constexpr double kMaxLoad = 0.5;                                // visited-table load limit
constexpr uint64_t kExactAllocLimit = 24ull << 30;  // allocate |<S>| states up front below this

// ---- allocator ------------------------------------------------------------------------
struct Allocator {
    cg_alloc_fn alloc = nullptr;
    cg_free_fn free_fn = nullptr;
    void* ctx = nullptr;
} g_alloc;

std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t pool_for(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) {
            cudaGetLastError();
            g_pool[dev] = nullptr;
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return g_pool[dev];
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (g_alloc.alloc) return g_alloc.alloc(bytes, st, g_alloc.ctx);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    cudaMemPool_t pool = pool_for(dev);
    if (!pool) return nullptr;
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, pool, st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, cudaStream_t st) {
    if (!p) return;
    if (g_alloc.free_fn) g_alloc.free_fn(p, st, g_alloc.ctx);
    else cudaFreeAsync(p, st);
}

// ---- generators -------------------------------------------------------------------------
bool is_perm_row(const uint8_t* g, int n) {   // n <= 128
    uint64_t seen[2] = {0, 0};
    for (int i = 0; i < n; ++i) {
        if (g[i] >= n || (seen[g[i] >> 6] >> (g[i] & 63)) & 1ull) return false;
        seen[g[i] >> 6] |= 1ull << (g[i] & 63);
    }
    return true;
}

bool is_identity_row(const uint8_t* g, int n) {
    for (int i = 0; i < n; ++i)
        if (g[i] != i) return false;
    return true;
}

// Device form of the gather t[i] = s[g[i]] on keys of w-bit elements (see GenSM): shift-and-mask
// terms, or, when those would be more than kMaxTerms, a range reversal if g reverses one
// contiguous range of positions and fixes the rest.  Returns false if neither form fits.
bool make_gensm_checked(const uint8_t* g, int n, int w, GenSM& G) {
    std::memset(&G, 0, sizeof(G));
    G.width = (uint8_t)w;
    const uint64_t elem_mask = (1ull << w) - 1;
    bool fits = true;
    for (int i = 0; i < n && fits; ++i) {
        const unsigned rot = (unsigned)(((w * (i - (int)g[i])) % 64 + 64) & 63);
        uint32_t t = 0;
        while (t < G.nterms && G.rot[t] != rot) ++t;
        if (t == G.nterms) {
            if (G.nterms == (uint32_t)cg::kMaxTerms) { fits = false; break; }
            G.rot[t] = (uint8_t)rot;
            G.nterms++;
        }
        G.mask[t] |= elem_mask << (w * i);
    }
    if (fits) return true;
    int a = -1, b = -1;
    for (int i = 0; i < n; ++i)
        if (g[i] != i) {
            if (a < 0) a = i;
            b = i;
        }
    bool reversal = a >= 0 && b > a;
    for (int i = a; reversal && i <= b; ++i) reversal = g[i] == a + b - i;
    if (!reversal) return false;
    std::memset(&G, 0, sizeof(G));
    G.width = (uint8_t)w;
    const int elems = 64 / w;   // after the bit reversal element e sits at elems - 1 - e
    G.kind = 1;
    G.rev_shift = (int16_t)(w * (elems - 1 - a - b));
    const uint64_t lo = (uint64_t)w * a, hi = (uint64_t)w * (b + 1);
    G.mask[0] = (hi >= 64 ? ~0ull : ((1ull << hi) - 1)) & ~((1ull << lo) - 1);
    return true;
}

// The same forms over two-word keys (WideGen): shift-and-mask over 128 bits with at most
// kMaxWideTerms terms, else the reversal of one contiguous range (widths 1, 2, 4, whose
// elements tile the 128 bits).  Returns false if neither fits.
bool make_widegen_checked(const uint8_t* g, int n, int w, cg::WideGen& G) {
    std::memset(&G, 0, sizeof(G));
    G.width = (uint8_t)w;
    bool fits = true;
    for (int i = 0; i < n && fits; ++i) {
        const unsigned rot = (unsigned)(((w * (i - (int)g[i])) % 128 + 128) & 127);
        uint32_t t = 0;
        while (t < G.nterms && G.rot[t] != rot) ++t;
        if (t == G.nterms) {
            if (G.nterms == (uint32_t)cg::kMaxWideTerms) { fits = false; break; }
            G.rot[t] = (uint8_t)rot;
            G.nterms++;
        }
        for (int b = 0; b < w; ++b) {
            const int bit = w * i + b;
            if (bit < 64) G.mlo[t] |= 1ull << bit;
            else G.mhi[t] |= 1ull << (bit - 64);
        }
    }
    if (fits) return true;
    if (w != 1 && w != 2 && w != 4) return false;
    int a = -1, b = -1;
    for (int i = 0; i < n; ++i)
        if (g[i] != i) {
            if (a < 0) a = i;
            b = i;
        }
    bool reversal = a >= 0 && b > a;
    for (int i = a; reversal && i <= b; ++i) reversal = g[i] == a + b - i;
    if (!reversal) return false;
    std::memset(&G, 0, sizeof(G));
    G.width = (uint8_t)w;
    G.kind = 1;
    const int elems = 128 / w;   // after the bit reversal element e sits at elems - 1 - e
    G.rev_shift = (int16_t)(w * (elems - 1 - a - b));
    for (int bit = w * a; bit < w * (b + 1); ++bit) {
        if (bit < 64) G.mlo[0] |= 1ull << bit;
        else G.mhi[0] |= 1ull << (bit - 64);
    }
    return true;
}

GenSM make_gensm(const uint8_t* g, int n, int w = 4) {
    GenSM G;
    make_gensm_checked(g, n, w, G);
    return G;
}

// Distinct non-identity rows.
std::vector<std::vector<uint8_t>> clean_rows(int n, int k, const uint8_t* gens) {
    std::set<std::vector<uint8_t>> seen;
    std::vector<std::vector<uint8_t>> out;
    for (int j = 0; j < k; ++j) {
        std::vector<uint8_t> r(gens + (size_t)j * n, gens + (size_t)(j + 1) * n);
        if (is_identity_row(r.data(), n)) continue;
        if (seen.insert(r).second) out.push_back(r);
    }
    return out;
}

// Shift-and-mask forms of distinct rows, with each generator's inverse tag (1 + index of its
// inverse among the rows when that index is below 15, else 0).
std::vector<GenSM> make_gensms(const std::vector<std::vector<uint8_t>>& rows, int n, int w = 4) {
    std::vector<GenSM> out;
    for (auto& r : rows) out.push_back(make_gensm(r.data(), n, w));
    for (size_t j = 0; j < rows.size(); ++j) {
        std::vector<uint8_t> inv(n);
        for (int i = 0; i < n; ++i) inv[rows[j][i]] = (uint8_t)i;
        for (size_t m = 0; m < rows.size() && m < 15; ++m)
            if (rows[m] == inv) { out[j].inv_tag = (uint32_t)(m + 1); break; }
    }
    return out;
}

// Two-word forms of distinct rows with the inverse tags (as make_gensms); false if a row fits
// neither form.
bool make_widegens(const std::vector<std::vector<uint8_t>>& rows, int n, int w, std::vector<cg::WideGen>& out) {
    out.assign(rows.size(), cg::WideGen{});
    for (size_t j = 0; j < rows.size(); ++j)
        if (!make_widegen_checked(rows[j].data(), n, w, out[j])) return false;
    for (size_t j = 0; j < rows.size(); ++j) {
        std::vector<uint8_t> inv(n);
        for (int i = 0; i < n; ++i) inv[rows[j][i]] = (uint8_t)i;
        for (size_t m = 0; m < rows.size() && m < 15; ++m)
            if (rows[m] == inv) { out[j].inv_tag = (uint32_t)(m + 1); break; }
    }
    return true;
}

bool closed_under_inverse(const std::vector<std::vector<uint8_t>>& rows, int n) {
    std::set<std::vector<uint8_t>> s(rows.begin(), rows.end());
    for (auto& r : rows) {
        std::vector<uint8_t> inv(n);
        for (int i = 0; i < n; ++i) inv[r[i]] = (uint8_t)i;
        if (!s.count(inv)) return false;
    }
    return true;
}

int validate(int n, int k, const uint8_t* gens, int max_n = cg::kMaxN) {
    if (n < 1 || n > max_n || k < 1 || gens == nullptr) return CG_EINVAL;
    for (int j = 0; j < k; ++j)
        if (!is_perm_row(gens + (size_t)j * n, n)) return CG_EINVAL;
    return CG_OK;
}

size_t al_up(size_t x) { return (x + 255) & ~size_t(255); }

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

uint64_t table_slots_for(uint64_t cap) {
    return std::max<uint64_t>(1024, next_pow2((uint64_t)((double)cap / kMaxLoad) + 1));
}

uint64_t bytes_for(uint64_t cap) { return cap * 8 + table_slots_for(cap) * 8; }

uint64_t factorial(int n) {
    uint64_t f = 1;
    for (int i = 2; i <= n; ++i) f *= (uint64_t)i;
    return f;
}

// Sweep strategy layout over S_n: 1024-rank blocks, and the bytes of V, two layer bitmaps,
// their block bits and block lists.
uint64_t sweep_blocks(int n) { return (factorial(n) + 1023) / 1024; }
uint64_t sweep_bytes(int n) {
    const uint64_t nb = sweep_blocks(n);
    const uint64_t words = nb * 32, sum = (nb + 31) / 32;
    return 4 * (3 * words + 2 * sum + 2 * nb) + 4096;
}

// 32-bit words of a rank bitmap over S_n, rounded up to whole 8-byte slots.
uint64_t bitmap_words(int n) { return ((factorial(n) + 63) / 64) * 2; }

// The rank bitmap (one bit per element of S_n) replaces the hash table when it fits and is not
// much larger than a table for the group: n <= 14, at most half of mem_cap and 16 GiB, and the
// group fills at least 1/512 of S_n.
bool bitmap_fits(int n, uint64_t mem) {
    if (n < 2 || n > 14) return false;
    const uint64_t bytes = bitmap_words(n) * 4;
    return bytes <= mem / 2 && bytes <= (16ull << 30);
}

bool bitmap_eligible(int n, uint64_t order, uint64_t mem) {
    return bitmap_fits(n, mem) && order * 512 >= factorial(n);
}

// Largest state capacity whose keys + table fit in `mem` bytes.
uint64_t max_cap_for_mem(uint64_t mem) {
    uint64_t best = 0;
    for (int p = 10; p <= 42; ++p) {
        const uint64_t slots = 1ull << p;
        if (slots * 8 >= mem) break;
        const uint64_t by_load = (uint64_t)((double)slots * kMaxLoad) - 1;
        const uint64_t by_mem = (mem - slots * 8) / 8;
        best = std::max(best, std::min(by_load, by_mem));
    }
    return best;
}

// The last CUDA error this thread turned into a return code, and the source line that did
// (cg_last_error_detail).
thread_local cudaError_t g_last_cuda_error = cudaSuccess;
thread_local int g_last_cuda_line = 0;
thread_local char g_last_detail[96];

int cuda_rc_at(cudaError_t e, int line) {
    if (e == cudaSuccess) return CG_OK;
    g_last_cuda_error = e;
    g_last_cuda_line = line;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA;
}
#define cuda_rc(e) cuda_rc_at((e), __LINE__)

// Milliseconds between two recorded events, 0 if they cannot be compared; a failed query must
// not stay pending as this thread's last error (the next launch check would report it).
float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

int status_to_rc(int status) {
    switch (status) {
        case cg::kDone: return CG_OK;
        case cg::kTruncRadius: return CG_TRUNC_RADIUS;
        case cg::kTruncAbove: return CG_TRUNC_ABOVE;
        case cg::kNeedMem: return CG_TRUNC_MEMCAP;
        case cg::kRunning: return CG_EDEVICE;
        default: return CG_EDEVICE;
    }
}

int device_grid_cache[64][32][2] = {};

// Blocks of the persistent kernel that fit co-resident on device `dev` (variant: ILP 1..4, +8
// for whole-sector table probing, +16 for the rank bitmap; multi: several jobs per launch).
int grow_grid(int dev, int ilp, bool multi = false) {
    if (dev < 0 || dev >= 64 || ilp < 1 || ilp > 20) return 0;
    int& c = device_grid_cache[dev][ilp][multi ? 1 : 0];
    if (!c) c = cg::hash_grow_max_grid(dev, ilp, multi);
    return c;
}

// Generators probed together per thread.  Hash tables (random DRAM probes): all of them when
// k <= 4, else 4.  Rank bitmap (L2-resident, one atomic per probe): 1 -- measured fastest, and
// the only bitmap variant that fits 64 registers without spilling.
int default_ilp(int k, bool bitmap = false) { return bitmap ? 1 : std::max(1, std::min(4, k)); }

}  // namespace

// ---- single job ---------------------------------------------------------------------------
struct cg_growth {
    int n = 0;
    int k = 0;                                   // distinct non-identity generators
    std::vector<GenSM> gsm;
    int inverse_closed = 0;
    int max_radius = -1;
    uint64_t mem_cap = kDefaultMemCap;
    int strategy = CG_STRATEGY_AUTO;
    uint64_t stop_above = 0;
    int keep_last = 0;
    int grid_override = 0;
    int ilp_override = 0;
    int sweep_order = 0;                         // CG_OPT_SWEEP_ORDER
    int mode = -1;                               // visited set chosen at the first run
    std::vector<std::vector<uint8_t>> rows;      // the distinct non-identity generators
    int width = 4;                               // bits per element of the packed keys
    bool wide = false;                           // n * width > 64: two-word keys (wide_path.cu)
    std::vector<cg::WideGen> wgsm;
    cg::Key128 wstart{0, 0};
    bool use_start = false;                      // grow from a central state instead of e
    bool start_constant = false;                 // every value of the start vector is the same
    uint64_t start_key = 0;
    bool start_is_perm = true;                   // the start vector has distinct entries
    uint64_t states_bound = 1;                   // states the growth can reach (orbit bound)
    uint64_t order = 1;
    int device = -1;
    cudaStream_t alloc_stream = nullptr;

    GenSM* d_gens = nullptr;
    JobDev* d_job = nullptr;
    Ctl* d_ctl = nullptr;
    unsigned long long* d_ubeg = nullptr;
    uint64_t* d_layers = nullptr;
    uint64_t* d_keys = nullptr;
    uint64_t keys_cap = 0;
    uint64_t* d_table = nullptr;
    uint64_t table_slots = 0;

    // sort strategy: three rotating sorted layers, candidate buffer, primitive scratch
    uint64_t* d_L[3] = {nullptr, nullptr, nullptr};
    uint64_t L_caps[3] = {0, 0, 0};
    uint64_t L_cap = 0;                          // largest of L_caps (reported in the stats)
    uint64_t* d_cand = nullptr;
    uint64_t cand_cap = 0;
    void* d_sort_scratch = nullptr;
    unsigned long long* d_count = nullptr;
    cg::SmallSteps* d_small = nullptr;           // state of the one-block small layer steps
    uint64_t* last_layer_ptr = nullptr;   // device pointer of the last reported layer
    uint64_t last_layer_n = 0;
    std::vector<uint64_t> sort_layers;

    // two-word keys: generators, descriptor, states, visited table of 16-byte slots
    cg::WideGen* d_wgens = nullptr;
    cg::WideDev* d_wjob = nullptr;
    cg::Key128* d_wkeys = nullptr;
    uint64_t wkeys_cap = 0;
    cg::Key128* d_wtable = nullptr;
    uint64_t wtable_slots = 0;
    cg::WideDev host_wide{};

    // sweep strategy: visited bitmap, two layer bitmaps with block bits and block lists
    SweepDev* d_sweep = nullptr;
    unsigned* d_sw = nullptr;                    // one allocation holding all of the below
    uint64_t sw_bytes = 0;
    SweepDev host_sweep{};
    bool last_is_sweep = false;

    JobDev host_job{};
    bool have_last = false;
    cg_growth_stats stats{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    void release(cudaStream_t st) {
        dev_free(d_gens, st);
        dev_free(d_job, st);
        dev_free(d_ctl, st);
        dev_free(d_ubeg, st);
        dev_free(d_layers, st);
        dev_free(d_keys, st);
        dev_free(d_table, st);
        d_gens = nullptr; d_job = nullptr; d_ctl = nullptr; d_ubeg = nullptr;
        d_layers = nullptr; d_keys = nullptr; d_table = nullptr;
        keys_cap = table_slots = 0;
        dev_free(d_sweep, st);
        dev_free(d_sw, st);
        d_sweep = nullptr;
        d_sw = nullptr;
        sw_bytes = 0;
        dev_free(d_wgens, st);
        dev_free(d_wjob, st);
        dev_free(d_wkeys, st);
        dev_free(d_wtable, st);
        d_wgens = nullptr; d_wjob = nullptr; d_wkeys = nullptr; d_wtable = nullptr;
        wkeys_cap = wtable_slots = 0;
        release_sort(st);
        have_last = false;                 // the last layer lived in the freed buffers
        last_layer_ptr = nullptr;
        last_layer_n = 0;
    }

    void release_sort(cudaStream_t st) {
        for (auto& p : d_L) { dev_free(p, st); p = nullptr; }
        for (auto& c : L_caps) c = 0;
        dev_free(d_cand, st);
        dev_free(d_sort_scratch, st);
        dev_free(d_count, st);
        dev_free(d_small, st);
        d_cand = nullptr; d_sort_scratch = nullptr; d_count = nullptr; d_small = nullptr;
        L_cap = cand_cap = 0;
    }
};

namespace {

int ensure_small_buffers(cg_growth* h, cudaStream_t st) {
    if (h->d_job) return CG_OK;
    h->d_gens = (GenSM*)dev_alloc(sizeof(GenSM) * std::max(1, h->k), st);
    h->d_job = (JobDev*)dev_alloc(sizeof(JobDev), st);
    h->d_ctl = (Ctl*)dev_alloc(sizeof(Ctl), st);
    h->d_ubeg = (unsigned long long*)dev_alloc(sizeof(unsigned long long) * 2, st);
    h->d_layers = (uint64_t*)dev_alloc(sizeof(uint64_t) * cg::kMaxLayers, st);
    if (!h->d_gens || !h->d_job || !h->d_ctl || !h->d_ubeg || !h->d_layers) return CG_ENOMEM;
    if (h->k > 0 && (int)h->gsm.size() == h->k) {   // one-word forms (two-word keys: none)
        cudaError_t e = cudaMemcpyAsync(h->d_gens, h->gsm.data(), sizeof(GenSM) * h->k,
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    return CG_OK;
}

// (Re)allocate keys + table for `cap` states, keeping the first `keep` keys.
int resize_state(cg_growth* h, uint64_t cap, uint64_t keep, cudaStream_t st) {
    uint64_t* keys = (uint64_t*)dev_alloc(cap * 8, st);
    if (!keys) return CG_ENOMEM;
    if (h->mode == cg::kVisitBitmap) {   // the bitmap has a fixed size: allocate it once
        if (!h->d_table) {
            h->table_slots = bitmap_words(h->n) / 2;
            h->d_table = (uint64_t*)dev_alloc(h->table_slots * 8, st);
            if (!h->d_table) { dev_free(keys, st); return CG_ENOMEM; }
        }
        if (keep > 0) {
            cudaError_t e = cudaMemcpyAsync(keys, h->d_keys, keep * 8, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) { dev_free(keys, st); return cuda_rc(e); }
        }
        dev_free(h->d_keys, st);
        h->d_keys = keys;
        h->keys_cap = cap;
        return CG_OK;
    }
    const uint64_t slots = table_slots_for(cap);
    uint64_t* table = (uint64_t*)dev_alloc(slots * 8, st);
    if (!table) { dev_free(keys, st); return CG_ENOMEM; }
    if (keep > 0) {
        cudaError_t e = cudaMemcpyAsync(keys, h->d_keys, keep * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { dev_free(keys, st); dev_free(table, st); return cuda_rc(e); }
    }
    dev_free(h->d_keys, st);
    dev_free(h->d_table, st);
    h->d_keys = keys;
    h->d_table = table;
    h->keys_cap = cap;
    h->table_slots = slots;
    return CG_OK;
}

void fill_static(cg_growth* h, JobDev& J) {
    J.keys = h->d_keys;
    J.keys_cap = h->keys_cap;
    J.table = h->d_table;
    J.table_mask = h->table_slots - 1;
    J.gens = h->d_gens;
    J.layer_sizes = h->d_layers;
    J.stop_above = h->stop_above;
    J.k = h->k;
    J.n = h->n;
    J.layers_cap = cg::kMaxLayers;
    J.max_radius = h->max_radius;
    J.mode = h->mode;
    J.bitmap_words = h->mode == cg::kVisitBitmap ? bitmap_words(h->n) : 0;
    J.use_start = h->use_start ? 1 : 0;
    J.start_key = h->start_key;
    J.tagged = h->n * h->width <= 60 ? 1 : 0;
    J.closed = 1;
    for (const GenSM& g : h->gsm) J.closed &= g.inv_tag != 0 ? 1 : 0;
}

int run_hash(cg_growth* h, cudaStream_t st, int* final_status) {
    // buffers of an earlier run that switched to the sorted step are not needed
    if (h->d_cand || h->d_L[0]) h->release_sort(st);
    const bool fresh_alloc = (h->d_job == nullptr);
    int rc = ensure_small_buffers(h, st);
    if (rc) return rc;
    if (fresh_alloc) h->stats.h2d_bytes += sizeof(GenSM) * h->k;
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    if (h->mode < 0) {
        // the rank bitmap indexes permutations: a start vector with repeated entries needs the
        // hash table
        if (h->strategy == CG_STRATEGY_BITMAP && (!bitmap_fits(h->n, mem) || !h->start_is_perm))
            return CG_EINVAL;
        h->mode = (h->strategy == CG_STRATEGY_BITMAP ||
                   (h->strategy == CG_STRATEGY_AUTO && h->start_is_perm &&
                    bitmap_eligible(h->n, h->order, mem)))
                      ? cg::kVisitBitmap : cg::kVisitHash;
    }
    const bool bitmap = h->mode == cg::kVisitBitmap;
    const int ilp = (h->ilp_override > 0 ? h->ilp_override : default_ilp(h->k, bitmap)) + (bitmap ? 16 : 0);
    const uint64_t avail = mem > (1 << 20) ? mem - (1 << 20) : mem;
    const uint64_t bm_bytes = bitmap ? bitmap_words(h->n) * 4 : 0;
    const uint64_t max_cap = std::min<uint64_t>(
        h->states_bound, bitmap ? (avail > bm_bytes ? (avail - bm_bytes) / 8 : 0) : max_cap_for_mem(avail));
    if (max_cap < 1) return CG_ENOMEM;
    if (!h->d_keys) {
        uint64_t start = h->states_bound;
        const uint64_t need = bitmap ? start * 8 + bm_bytes : bytes_for(start);
        if (need > std::min<uint64_t>(mem, kExactAllocLimit))
            start = std::min<uint64_t>(max_cap, 1ull << 24);
        start = std::min(start, max_cap);
        rc = resize_state(h, std::max<uint64_t>(start, 1), 0, st);
        if (rc) return rc;
    }
    const int grid_max = grow_grid(h->device, ilp);
    if (grid_max <= 0) return CG_ECUDA;
    // Small groups finish faster with fewer blocks at each barrier.
    const uint64_t want = h->states_bound / (32 * 8 * 2) + 1;
    int grid = (int)std::min<uint64_t>((uint64_t)grid_max, std::max<uint64_t>(want, 1));
    if (h->grid_override > 0) grid = std::min(grid_max, h->grid_override);

    cudaError_t e = cudaMemsetAsync(h->d_table, bitmap ? 0 : 0xFF, h->table_slots * 8, st);
    if (e != cudaSuccess) return cuda_rc(e);
    JobDev J;
    std::memset(&J, 0, sizeof(J));
    fill_static(h, J);
    if ((e = cudaMemcpyAsync(h->d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cg::launch_init_jobs(h->d_job, 1, h->d_ubeg, h->d_ctl, st)) != cudaSuccess)
        return cuda_rc(e);
    h->stats.launches += 2;  // init_jobs + init_units
    h->stats.h2d_bytes += sizeof(J);
    if (!h->ev0) {
        if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return cuda_rc(e);
    }
    // A rank bitmap larger than L2 takes its random atomics from DRAM.  Keys in ascending order are
    // in Lehmer-rank order (the value at position n - 1 is the top rank digit, and so on down), and
    // a generator that moves only positions below j sends a state within j! ranks of it: a frontier
    // grouped by its top four elements keeps the visited words of most images inside the group's
    // stretch of the bitmap, which L2 holds while the grid works through it.  Such a growth runs
    // one round per launch, and a frontier of at least kOrderMinStates states is first put in order
    // of key bits [4n - 16, 4n) (two stable 8-bit passes; the parent-edge tags ride along), when
    // the sort's scratch fits beside the job's buffers within mem_cap.
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) {
        (void)cudaGetLastError();
        l2 = 0;
    }
    const bool order_frontier = bitmap && h->start_is_perm && h->width == 4 && h->n >= 8 && l2 > 0 &&
                                bm_bytes > (uint64_t)l2;
    for (;;) {
        if ((e = cudaEventRecord(h->ev0, st)) != cudaSuccess) return cuda_rc(e);
        int sort_err = 0;
        if (order_frontier) {
            const uint64_t F = J.hi > J.lo ? J.hi - J.lo : 0;
            const uint64_t need = cg::sort_scratch_bytes(F);
            if (F >= kOrderMinStates && h->keys_cap * 8 + bm_bytes + need <= mem) {
                void* scr = dev_alloc(need, st);
                if (scr) {
                    const cg::SortScratch sc = cg::carve_sort_scratch(scr, F);
                    e = cudaMemsetAsync(sc.err, 0, 4, st);
                    if (e == cudaSuccess)
                        e = cg::launch_radix_sort(h->d_keys + J.lo, F, 4 * h->n, sc, st, 4 * h->n - 16);
                    if (e == cudaSuccess) e = cudaMemcpyAsync(&sort_err, sc.err, 4, cudaMemcpyDeviceToHost, st);
                    dev_free(scr, st);
                    if (e != cudaSuccess) return cuda_rc(e);
                    h->stats.launches += 1 + cg::sort_passes(4 * h->n, 4 * h->n - 16);
                    h->stats.d2h_bytes += 4;
                }
            }
        }
        if ((e = cg::launch_hash_grow(h->d_job, 1, h->d_ubeg, h->d_ctl, grid,
                                      order_frontier ? 1 : cg::kMaxLayers + 1, kTimeoutNs, ilp, st, h->n,
                                      nullptr, &J)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaEventRecord(h->ev1, st)) != cudaSuccess) return cuda_rc(e);
        h->stats.launches += 1;
        Ctl ctl;
        if ((e = cudaMemcpyAsync(&J, h->d_job, sizeof(J), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaMemcpyAsync(&ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
        h->stats.d2h_bytes += sizeof(J) + sizeof(ctl);
        h->stats.kernel_ms += elapsed_ms(h->ev0, h->ev1);
        h->stats.rounds += ctl.rounds;
        if (ctl.err) return ctl.err;
        if (sort_err) return sort_err;
        if (order_frontier && J.status == cg::kRunning) {
            // the next round, in its own launch
            if ((e = cg::launch_resume_units(h->d_job, 1, h->d_ubeg, h->d_ctl, st)) != cudaSuccess)
                return cuda_rc(e);
            h->stats.launches += 1;
            continue;
        }
        if (J.status != cg::kNeedMem) break;
        if (h->keys_cap >= max_cap) break;  // cannot grow: truncated by mem_cap
        // Grow: keep layers 0..radius (keys[0, hi)), rebuild the visited table from them.
        const uint64_t keep = J.hi;
        const uint64_t newcap = std::min<uint64_t>(max_cap, std::max<uint64_t>(h->keys_cap * 4, keep + 1));
        if ((rc = resize_state(h, newcap, keep, st))) return rc;
        if ((e = cudaMemsetAsync(h->d_table, bitmap ? 0 : 0xFF, h->table_slots * 8, st)) != cudaSuccess)
            return cuda_rc(e);
        e = bitmap ? cg::launch_rebuild_bitmap(h->d_keys, keep, reinterpret_cast<unsigned*>(h->d_table),
                                               bitmap_words(h->n), h->n, &h->d_ctl->err, grid_max, st)
                   : cg::launch_rebuild_table(h->d_keys, keep, h->d_table, h->table_slots - 1,
                                              h->n * h->width <= 60 ? cg::kKeyBits60 : ~0ull, &h->d_ctl->err,
                                              grid_max, st);
        if (e != cudaSuccess) return cuda_rc(e);
        fill_static(h, J);
        J.tail = J.hi;
        J.overflow = 0;
        J.status = cg::kRunning;
        if ((e = cudaMemcpyAsync(h->d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cg::launch_resume_units(h->d_job, 1, h->d_ubeg, h->d_ctl, st)) != cudaSuccess)
            return cuda_rc(e);
        h->stats.launches += 2;  // rebuild_table + init_units
        h->stats.h2d_bytes += sizeof(J);
    }
    h->stats.state_capacity = h->keys_cap;
    h->stats.table_slots = h->table_slots;
    h->stats.strategy_used = bitmap ? CG_STRATEGY_BITMAP : CG_STRATEGY_HASH;
    h->stats.probe_variant = ilp;
    h->host_job = J;
    *final_status = J.status;
    h->last_layer_ptr = h->d_keys + J.lo;
    h->last_layer_n = J.hi - J.lo;
    return CG_OK;
}

// ---- two-word keys ---------------------------------------------------------------------------
// Vectors of more than 64 bits (wide_path.cu): one persistent launch; when the states or the
// visited table run out the host grows both x4 (within mem_cap), re-inserts the stored states
// and relaunches from the last complete layer, as run_hash does.

// (Re)allocate states and table for `cap` states keeping the first `keep` states.
int resize_wide(cg_growth* h, uint64_t cap, uint64_t keep, cudaStream_t st) {
    auto* keys = (cg::Key128*)dev_alloc(cap * 16, st);
    const uint64_t slots = table_slots_for(cap);
    auto* table = (cg::Key128*)dev_alloc(slots * 16, st);
    if (!keys || !table) { dev_free(keys, st); dev_free(table, st); return CG_ENOMEM; }
    if (keep > 0) {
        cudaError_t e = cudaMemcpyAsync(keys, h->d_wkeys, keep * 16, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { dev_free(keys, st); dev_free(table, st); return cuda_rc(e); }
    }
    dev_free(h->d_wkeys, st);
    dev_free(h->d_wtable, st);
    h->d_wkeys = keys;
    h->d_wtable = table;
    h->wkeys_cap = cap;
    h->wtable_slots = slots;
    return CG_OK;
}

int run_wide(cg_growth* h, cudaStream_t st, int* final_status) {
    if (h->strategy != CG_STRATEGY_AUTO && h->strategy != CG_STRATEGY_HASH) return CG_EINVAL;
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    const uint64_t avail = mem > (1 << 20) ? mem - (1 << 20) : mem;
    // 16 bytes a state plus 32 bytes of table (load <= 0.5), rounded to a power of two
    uint64_t max_cap = 0;
    for (int p = 10; p <= 40; ++p) {
        const uint64_t slots = 1ull << p;
        if (slots * 16 >= avail) break;
        max_cap = std::max(max_cap, std::min<uint64_t>((uint64_t)(slots * kMaxLoad) - 1, (avail - slots * 16) / 16));
    }
    max_cap = std::min(max_cap, h->states_bound);
    if (max_cap < 1) return CG_ENOMEM;
    int rc = ensure_small_buffers(h, st);
    if (rc) return rc;
    if (!h->d_wgens) {
        h->d_wgens = (cg::WideGen*)dev_alloc(sizeof(cg::WideGen) * std::max(1, h->k), st);
        h->d_wjob = (cg::WideDev*)dev_alloc(sizeof(cg::WideDev), st);
        if (!h->d_wgens || !h->d_wjob) return CG_ENOMEM;
        cudaError_t e = cudaMemcpyAsync(h->d_wgens, h->wgsm.data(), sizeof(cg::WideGen) * h->k,
                                        cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_rc(e);
        h->stats.h2d_bytes += sizeof(cg::WideGen) * h->k;
    }
    if (!h->d_wkeys) {
        uint64_t start = std::min<uint64_t>(max_cap, 1ull << 22);
        if (h->states_bound <= max_cap && h->states_bound * 48 <= std::min<uint64_t>(mem, kExactAllocLimit))
            start = h->states_bound;
        if ((rc = resize_wide(h, std::max<uint64_t>(start, 1), 0, st))) return rc;
    }
    const int tagged = h->n * h->width <= 124 ? 1 : 0;
    auto fill = [&](cg::WideDev& D) {
        D.keys = h->d_wkeys;
        D.keys_cap = h->wkeys_cap;
        D.table = h->d_wtable;
        D.table_mask = h->wtable_slots - 1;
        D.gens = h->d_wgens;
        D.layer_sizes = h->d_layers;
        D.stop_above = h->stop_above;
        D.start = h->wstart;
        D.k = h->k;
        D.n = h->n;
        D.layers_cap = cg::kMaxLayers;
        D.max_radius = h->max_radius;
        D.tagged = tagged;
    };
    cg::WideDev D;
    std::memset(&D, 0, sizeof(D));
    fill(D);
    cudaError_t e = cudaMemsetAsync(h->d_wtable, 0xFF, h->wtable_slots * 16, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_wjob, &D, sizeof(D), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), st);
    if (e == cudaSuccess) e = cg::launch_wide_init(h->d_wjob, st);
    if (e != cudaSuccess) return cuda_rc(e);
    h->stats.launches += 1;
    h->stats.h2d_bytes += sizeof(D);
    if (!h->ev0) {
        if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return cuda_rc(e);
    }
    const int grid_max = cg::wide_max_grid(h->device);
    if (grid_max <= 0) return CG_ECUDA;
    int grid = (int)std::min<uint64_t>((uint64_t)grid_max, h->states_bound / 512 + 1);
    if (h->grid_override > 0) grid = std::min(grid_max, h->grid_override);
    for (;;) {
        if ((e = cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), st)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaEventRecord(h->ev0, st)) != cudaSuccess) return cuda_rc(e);
        if ((e = cg::launch_wide_grow(h->d_wjob, h->d_ctl, grid, cg::kMaxLayers + 1, kTimeoutNs, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaEventRecord(h->ev1, st)) != cudaSuccess) return cuda_rc(e);
        h->stats.launches += 1;
        Ctl ctl;
        if ((e = cudaMemcpyAsync(&D, h->d_wjob, sizeof(D), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaMemcpyAsync(&ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
        h->stats.d2h_bytes += sizeof(D) + sizeof(ctl);
        h->stats.kernel_ms += elapsed_ms(h->ev0, h->ev1);
        h->stats.rounds += ctl.rounds;
        if (ctl.err) return ctl.err;
        if (D.status != cg::kNeedMem) break;
        if (h->wkeys_cap >= max_cap) break;   // cannot grow: truncated by mem_cap
        const uint64_t keep = D.hi;
        const uint64_t newcap = std::min<uint64_t>(max_cap, std::max<uint64_t>(h->wkeys_cap * 4, keep + 1));
        if ((rc = resize_wide(h, newcap, keep, st))) return rc;
        if ((e = cudaMemsetAsync(h->d_wtable, 0xFF, h->wtable_slots * 16, st)) != cudaSuccess) return cuda_rc(e);
        if ((e = cg::launch_wide_rebuild(h->d_wkeys, keep, h->d_wtable, h->wtable_slots - 1, tagged,
                                         &h->d_ctl->err, grid_max, st)) != cudaSuccess)
            return cuda_rc(e);
        fill(D);
        D.tail = D.hi;
        D.overflow = 0;
        D.status = cg::kRunning;
        if ((e = cudaMemcpyAsync(h->d_wjob, &D, sizeof(D), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
        int derr = 0;
        if ((e = cudaMemcpy(&derr, &h->d_ctl->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_rc(e);
        if (derr) return derr;
        h->stats.launches += 1;
        h->stats.h2d_bytes += sizeof(D);
    }
    h->stats.state_capacity = h->wkeys_cap;
    h->stats.table_slots = h->wtable_slots;
    h->stats.strategy_used = CG_STRATEGY_HASH;
    h->stats.probe_variant = 1;
    h->host_wide = D;
    std::memset(&h->host_job, 0, sizeof(h->host_job));
    h->host_job.radius = D.radius;
    h->host_job.status = D.status;
    *final_status = D.status;
    return CG_OK;
}

// ---- sweep strategy driver -----------------------------------------------------------------
// Bitmaps over S_n for the visited set and two layers (sweep_path.cu: 3 bits per element); one
// persistent launch runs every layer step.  Needs a start with distinct values and n <= 14.

// AUTO takes the sweep for the whole growth (no radius or layer-size limit) of a dense subgroup
// of S_n whose states, stored as keys beside a rank bitmap, would not fit the memory cap while
// the sweep's bitmaps do.  With a limit the key-list path runs first: it is faster while the
// states it stores fit, and grows its buffers as the layers come.
bool sweep_preferred(const cg_growth* h) {
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    if (!h->start_is_perm || h->n > 14 || h->n < 2) return false;
    if (h->max_radius >= 0 || h->stop_above > 0) return false;
    if (h->order * 512 < factorial(h->n)) return false;
    if (sweep_bytes(h->n) > mem) return false;
    return h->states_bound * 8 + bitmap_words(h->n) * 4 > mem;
}

int run_sweep(cg_growth* h, cudaStream_t st, int* final_status) {
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    if (!h->start_is_perm || h->n > 14 || h->n < 1) return CG_EINVAL;
    const uint64_t bytes = sweep_bytes(h->n);
    if (bytes > mem) return CG_EINVAL;
    int rc = ensure_small_buffers(h, st);
    if (rc) return rc;
    const uint64_t nb = sweep_blocks(h->n);
    const uint64_t words = nb * 32, nsum = (nb + 31) / 32;
    if (!h->d_sw) {
        h->d_sw = (unsigned*)dev_alloc(bytes, st);
        h->d_sweep = (SweepDev*)dev_alloc(sizeof(SweepDev), st);
        if (!h->d_sw || !h->d_sweep) return CG_ENOMEM;
        h->sw_bytes = bytes;
    }
    // layout: V | F0 F1 | S0 S1 | L0 L1   (32-bit words)
    SweepDev D;
    std::memset(&D, 0, sizeof(D));
    unsigned* p = h->d_sw;
    D.V = p; p += words;
    for (int i = 0; i < 2; ++i) { D.F[i] = p; p += words; }
    for (int i = 0; i < 2; ++i) { D.S[i] = p; p += nsum; }
    for (int i = 0; i < 2; ++i) { D.L[i] = p; p += nb; }
    D.gens = h->d_gens;
    D.layer_sizes = h->d_layers;
    D.nblocks = nb;
    D.stop_above = h->stop_above;
    D.k = h->k;
    D.n = h->n;
    D.layers_cap = cg::kMaxLayers;
    D.max_radius = h->max_radius < 0 ? -1 : h->max_radius;
    // rank of the start (identity: 0), position-major Lehmer digits taken from the top down
    {
        uint8_t v[16];
        for (int i = 0; i < h->n; ++i)
            v[i] = h->use_start ? (uint8_t)((h->start_key >> (4 * i)) & 15u) : (uint8_t)i;
        uint64_t r = 0;
        unsigned right = 0;
        for (int i = h->n - 1; i >= 1; --i) {
            unsigned d = v[i];
            for (unsigned u = 0; u < v[i]; ++u) d -= (right >> u) & 1u;
            right |= 1u << v[i];
            r = r * (uint64_t)(i + 1) + d;
        }
        D.start_rank = r;
    }
    // V, F and S start empty (the lists need no clearing: lcount bounds them)
    cudaError_t e = cudaMemsetAsync(D.V, 0, (3 * words + 2 * nsum) * 4, st);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((e = cudaMemcpyAsync(h->d_sweep, &D, sizeof(D), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemsetAsync(h->d_ctl, 0, sizeof(Ctl), st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cg::launch_sweep_init(h->d_sweep, st)) != cudaSuccess) return cuda_rc(e);
    h->stats.launches += 1;
    h->stats.h2d_bytes += sizeof(D);
    // two generators in flight per thread measured best (S_12 Coxeter, S_13 pancake)
    const int ilp = h->ilp_override > 0 ? h->ilp_override : std::min(h->k, 2);
    int grid = cg::sweep_max_grid(h->device, ilp, h->n);
    if (grid <= 0) return CG_ECUDA;
    if (h->grid_override > 0) grid = std::min(grid, h->grid_override);
    if (!h->ev0) {
        if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return cuda_rc(e);
    }
    if ((e = cudaEventRecord(h->ev0, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cg::launch_sweep_grow(h->d_sweep, h->d_ctl, grid, cg::kMaxLayers + 1, kSweepTimeoutNs, ilp,
                                   h->n, h->sweep_order, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaEventRecord(h->ev1, st)) != cudaSuccess) return cuda_rc(e);
    h->stats.launches += 1;
    Ctl ctl;
    if ((e = cudaMemcpyAsync(&D, h->d_sweep, sizeof(D), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(&ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
    h->stats.d2h_bytes += sizeof(D) + sizeof(ctl);
    h->stats.kernel_ms += elapsed_ms(h->ev0, h->ev1);
    h->stats.rounds += ctl.rounds;
    if (ctl.err) return ctl.err;
    h->stats.state_capacity = factorial(h->n);
    h->stats.table_slots = words / 2;
    h->stats.strategy_used = CG_STRATEGY_SWEEP;
    h->stats.probe_variant = ilp;
    h->host_sweep = D;
    std::memset(&h->host_job, 0, sizeof(h->host_job));
    h->host_job.radius = D.radius;
    h->host_job.status = D.status;
    *final_status = D.status;
    return CG_OK;
}

// ---- sort strategy driver ------------------------------------------------------------------
// Layers live in three rotating buffers sorted ascending; each layer step is expand, radix
// sort, unique + merge-path difference against layers r and r-1, compaction (sort_path.cu).
// The host reads |L_{r+1}| after each step to size the next one.

// Bytes of the candidate buffer and sort scratch for q candidates.
uint64_t cand_bytes(uint64_t q) { return q * 8 + cg::sort_scratch_bytes(q); }

// First key bit the radix passes need: the states of a growth from a permutation are
// permutations, whose element at position 0 is the one value missing from the others, so two
// keys that agree above it are equal and ordering them on bits [w, w n) gives the order of the
// whole keys (one 8-bit pass fewer for n = 11).  Other vectors sort on all their bits.
int sort_low_bit(const cg_growth* h) { return h->start_is_perm && h->width == 4 ? 4 : 0; }

// Candidate buffer and scratch for q candidates (kept when larger, unless shrink).
int ensure_cand(cg_growth* h, uint64_t q, cudaStream_t st, bool shrink = false) {
    if (h->d_cand && (q == h->cand_cap || (q < h->cand_cap && !shrink))) return CG_OK;
    dev_free(h->d_cand, st);
    dev_free(h->d_sort_scratch, st);
    h->d_cand = (uint64_t*)dev_alloc(q * 8, st);
    h->d_sort_scratch = dev_alloc(cg::sort_scratch_bytes(q), st);
    h->cand_cap = q;
    if (!h->d_cand || !h->d_sort_scratch) return CG_ENOMEM;
    return CG_OK;
}

// Layer buffer i with room for cap keys, keeping its first `keep` keys.
int ensure_layer(cg_growth* h, int i, uint64_t cap, uint64_t keep, cudaStream_t st) {
    if (cap <= h->L_caps[i] && h->d_L[i]) return CG_OK;
    uint64_t* nb = (uint64_t*)dev_alloc(std::max<uint64_t>(cap, 1) * 8, st);
    if (!nb) return CG_ENOMEM;
    if (keep && h->d_L[i]) {
        cudaError_t e = cudaMemcpyAsync(nb, h->d_L[i], keep * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { dev_free(nb, st); return cuda_rc(e); }
    }
    dev_free(h->d_L[i], st);
    h->d_L[i] = nb;
    h->L_caps[i] = std::max<uint64_t>(cap, 1);
    h->L_cap = std::max(h->L_cap, h->L_caps[i]);
    return CG_OK;
}

// Layer steps of the sort strategy from layer `radius` (d_L[cur], Fcur keys) and layer radius-1
// (d_L[prev], Fprev keys), both sorted; sort_layers holds |L_0| .. |L_radius|.
//
// A step whose k Fcur candidates fit the memory cap at once is: candidate histograms + radix
// passes (expand fused, sorted candidates in d_cand), then first-of-run + difference against
// L_r and L_{r-1} + compaction into the scratch, copied into the next layer's buffer.  Larger
// steps run in key-range chunks: the top-digit histogram of all candidates splits the digit
// values into ranges of at most the candidate capacity; per range the candidates are generated
// again and kept when they fall in it, sorted, and differenced -- the ranges are disjoint and
// ascending, so their survivors append to layer r+1 in order.
int sort_steps(cg_growth* h, cudaStream_t st, int cur, int prev, uint64_t Fcur, uint64_t Fprev,
               int radius, int* final_status) {
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    const int bits = h->width * h->n;
    const int lo = sort_low_bit(h);
    const int P = cg::sort_passes(bits, lo);
    const int top_shift = lo + 8 * (P - 1);
    int nxt = 3 - cur - prev;
    cudaError_t e = cudaSuccess;
    int rc = CG_OK;
    if (!h->ev0) {
        if ((e = cudaEventCreate(&h->ev0)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaEventCreate(&h->ev1)) != cudaSuccess) return cuda_rc(e);
    }
    auto fail_mem = [](int r) { return r == CG_ENOMEM || r == CG_TRUNC_MEMCAP; };
    int status = cg::kRunning;
    while (status == cg::kRunning) {
        if (h->max_radius >= 0 && radius >= h->max_radius) { status = cg::kTruncRadius; break; }
        if ((uint64_t)h->k * Fcur <= (uint64_t)cg::kSmallStep && Fprev <= (uint64_t)cg::kSmallStep) {
            // small steps, back to back in one block (sort_path.cu): the three layer buffers
            // hold kSmallStep keys at least
            rc = ensure_layer(h, cur, cg::kSmallStep, Fcur, st);
            if (rc == CG_OK) rc = ensure_layer(h, prev, cg::kSmallStep, Fprev, st);
            if (rc == CG_OK) rc = ensure_layer(h, nxt, cg::kSmallStep, 0, st);
            if (rc == CG_OK && !h->d_small) {
                h->d_small = (cg::SmallSteps*)dev_alloc(sizeof(cg::SmallSteps), st);
                if (!h->d_small) rc = CG_ENOMEM;
            }
            if (fail_mem(rc)) { status = cg::kNeedMem; break; }
            if (rc) return rc;
            cg::SmallSteps ss{};
            ss.cur = cur;
            ss.prev = prev;
            ss.radius = radius;
            ss.status = cg::kRunning;
            ss.Fcur = Fcur;
            ss.Fprev = Fprev;
            const size_t head = offsetof(cg::SmallSteps, sizes);
            if ((e = cudaMemcpyAsync(h->d_small, &ss, head, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_rc(e);
            if ((e = cudaEventRecord(h->ev0, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cg::launch_small_steps(h->d_gens, h->k, h->d_L[0], h->d_L[1], h->d_L[2], h->max_radius,
                                            h->stop_above, (int)h->sort_layers.size(), h->d_small, st)) !=
                cudaSuccess)
                return cuda_rc(e);
            if ((e = cudaEventRecord(h->ev1, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaMemcpyAsync(&ss, h->d_small, sizeof(ss), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                return cuda_rc(e);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
            h->stats.launches += 1;
            h->stats.h2d_bytes += head;
            h->stats.d2h_bytes += sizeof(ss);
            h->stats.kernel_ms += elapsed_ms(h->ev0, h->ev1);
            h->stats.rounds += ss.nsteps;
            if (ss.nsteps < 0 || ss.nsteps > cg::kSmallMaxSteps || ss.cur < 0 || ss.cur > 2 || ss.prev < 0 ||
                ss.prev > 2 || ss.cur == ss.prev)
                return CG_EDEVICE;
            for (int i = 0; i < ss.nsteps; ++i) h->sort_layers.push_back(ss.sizes[i]);
            cur = ss.cur;
            prev = ss.prev;
            nxt = 3 - cur - prev;
            radius = ss.radius;
            Fcur = ss.Fcur;
            Fprev = ss.Fprev;
            status = ss.status;
            if (status != cg::kRunning) break;
            if (ss.nsteps > 0) continue;
        }
        const uint64_t C = (uint64_t)h->k * Fcur;
        // the next layer's first buffer: the growth ratio of the last step, with a margin
        const double ratio = Fprev > 0 ? (double)Fcur / (double)Fprev : (double)h->k;
        uint64_t est = (uint64_t)std::min<double>((double)C, std::max(1024.0, 1.2 * ratio * (double)Fcur));
        est = std::min<uint64_t>(est, h->states_bound);
        // the candidates' share of the memory cap, beside the three layers (held or planned)
        const uint64_t held_layers = 8 * (std::max(h->L_caps[cur], Fcur) + std::max(h->L_caps[prev], Fprev) +
                                          std::max(h->L_caps[nxt], est));
        if (held_layers + cand_bytes(4096) >= mem) { status = cg::kNeedMem; break; }
        uint64_t Q = std::min<uint64_t>(C, (mem - held_layers) * 2 / 33);   // 16.5 bytes a candidate
        while (Q > 4096 && held_layers + cand_bytes(Q) > mem) Q -= Q / 64 + 1;
        if (h->cand_cap >= C && held_layers + cand_bytes(h->cand_cap) <= mem) Q = C;   // allocated
        if (Q < std::min<uint64_t>(C, 4096)) { status = cg::kNeedMem; break; }
        // a larger buffer from an earlier step is kept while it fits beside the layers
        rc = ensure_cand(h, Q, st, held_layers + cand_bytes(h->cand_cap) > mem);
        if (rc == CG_OK) rc = ensure_layer(h, nxt, est, 0, st);
        if (fail_mem(rc)) { status = cg::kNeedMem; break; }
        if (rc) return rc;
        cg::SortScratch sc = cg::carve_sort_scratch(h->d_sort_scratch, h->cand_cap);
        const cg::ExpandSrc src{h->d_gens, h->k, h->d_L[cur], Fcur};
        const uint64_t* bs[2] = {h->d_L[cur], h->d_L[prev]};
        const unsigned long long nbs[2] = {Fcur, Fprev};
        if ((e = cudaMemsetAsync(sc.err, 0, 4, st)) != cudaSuccess) return cuda_rc(e);
        // key ranges of top-digit values [lo, hi): one range when everything fits
        std::vector<std::pair<unsigned, unsigned>> ranges;
        if (C <= h->cand_cap) {
            ranges.push_back({0u, 256u});
        } else {
            if ((e = cg::launch_candidate_hist(src, bits, sc, st, lo)) != cudaSuccess) return cuda_rc(e);
            std::vector<unsigned long long> th(256);
            if ((e = cudaMemcpyAsync(th.data(), sc.ghist + (size_t)(P - 1) * 256, 256 * 8, cudaMemcpyDeviceToHost,
                                     st)) != cudaSuccess)
                return cuda_rc(e);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
            h->stats.launches += 1;
            h->stats.d2h_bytes += 256 * 8;
            unsigned lo = 0;
            uint64_t acc = 0;
            bool ok = true;
            for (unsigned d = 0; d < 256 && ok; ++d) {
                if (th[d] > h->cand_cap) ok = false;            // one digit value alone is too many
                else if (acc + th[d] > h->cand_cap) { ranges.push_back({lo, d}); lo = d; acc = th[d]; }
                else acc += th[d];
            }
            if (!ok) { status = cg::kNeedMem; break; }
            ranges.push_back({lo, 256u});
        }
        uint64_t Fn = 0;
        bool stop_mem = false;
        for (const auto& rg : ranges) {
            if ((e = cudaEventRecord(h->ev0, st)) != cudaSuccess) return cuda_rc(e);
            uint64_t Cc = C;
            if (ranges.size() == 1) {
                if ((e = cg::launch_expand_sort(src, h->d_cand, bits, sc, st, lo)) != cudaSuccess) return cuda_rc(e);
                h->stats.launches += 1 + P;
            } else {
                if ((e = cg::launch_expand_filter(src, top_shift, rg.first, rg.second, h->d_cand, h->cand_cap,
                                                  h->d_count, sc.err, st)) != cudaSuccess)
                    return cuda_rc(e);
                unsigned long long got = 0;
                if ((e = cudaMemcpyAsync(&got, h->d_count, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
                    return cuda_rc(e);
                if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
                Cc = std::min<uint64_t>(got, h->cand_cap);
                if ((e = cg::launch_radix_sort(h->d_cand, Cc, bits, sc, st, lo)) != cudaSuccess) return cuda_rc(e);
                h->stats.launches += 2 + P;
            }
            if ((e = cg::launch_unique_difference(h->d_cand, Cc, bs, nbs, 2, sc.keys_tmp, h->d_count, sc, st)) !=
                cudaSuccess)
                return cuda_rc(e);
            if ((e = cudaEventRecord(h->ev1, st)) != cudaSuccess) return cuda_rc(e);
            h->stats.launches += 1;
            unsigned long long Fc = 0;
            int derr = 0;
            if ((e = cudaMemcpyAsync(&Fc, h->d_count, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaMemcpyAsync(&derr, sc.err, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
            h->stats.d2h_bytes += 12;
            h->stats.kernel_ms += elapsed_ms(h->ev0, h->ev1);
            if (derr) return derr;
            if (Fc == 0) continue;
            // append to the next layer, growing its buffer when the estimate was short
            if (Fn + Fc > h->L_caps[nxt]) {
                const uint64_t want = std::max<uint64_t>(Fn + Fc, h->L_caps[nxt] + h->L_caps[nxt] / 2);
                rc = ensure_layer(h, nxt, std::min<uint64_t>(want, std::max<uint64_t>(C, Fn + Fc)), Fn, st);
                if (fail_mem(rc)) { stop_mem = true; break; }
                if (rc) return rc;
            }
            if ((e = cudaMemcpyAsync(h->d_L[nxt] + Fn, sc.keys_tmp, Fc * 8, cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
                return cuda_rc(e);
            Fn += Fc;
        }
        h->stats.rounds += 1;
        if (stop_mem) { status = cg::kNeedMem; break; }
        if (Fn == 0) { status = cg::kDone; break; }
        h->sort_layers.push_back(Fn);
        ++radius;
        const int old_prev = prev;
        prev = cur;
        cur = nxt;
        nxt = old_prev;
        Fprev = Fcur;
        Fcur = Fn;
        if (h->stop_above > 0 && Fn > h->stop_above) { status = cg::kTruncAbove; break; }
        if ((int)h->sort_layers.size() >= cg::kMaxLayers) { status = cg::kTruncRadius; break; }
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
    h->host_job.radius = radius;
    h->host_job.status = status;
    h->last_layer_ptr = h->d_L[cur];
    h->last_layer_n = Fcur;
    h->stats.state_capacity = h->L_cap;
    h->stats.table_slots = 0;
    h->stats.strategy_used = CG_STRATEGY_SORT;
    h->stats.probe_variant = 0;
    *final_status = status;
    return CG_OK;
}

int run_sort(cg_growth* h, cudaStream_t st, int* final_status) {
    int rc = ensure_small_buffers(h, st);
    if (rc) return rc;
    if (!h->d_count) {
        h->d_count = (unsigned long long*)dev_alloc(64, st);
        if (!h->d_count) return CG_ENOMEM;
    }
    h->sort_layers.assign(1, 1);
    if ((rc = ensure_cand(h, std::max<uint64_t>((uint64_t)h->k, 4096), st))) return rc;
    if ((rc = ensure_layer(h, 0, 1, 0, st))) return rc;
    if ((rc = ensure_layer(h, 1, 1, 0, st))) return rc;
    uint64_t id = 0;
    for (int i = 0; i < h->n; ++i) id |= (uint64_t)i << (4 * i);
    if (h->use_start) id = h->start_key;
    cudaError_t e = cudaMemcpyAsync(h->d_L[0], &id, 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_rc(e);
    h->stats.h2d_bytes += 8;
    return sort_steps(h, st, 0, 1, 1, 0, 0, final_status);
}


// AUTO, undirected generating set: when the states stored by the visited-set path outgrow
// mem_cap, the growth goes on with the sorted layer step, which keeps only the last two layers
// (in an undirected graph the neighbours of layer r lie in layers r-1, r and r+1).  The visited
// set is released, layers L_{r-1} and L_r are copied on the device into the sorted step's layer
// buffers (while the key store still exists the job holds up to their size beyond what it held),
// stripped of their parent-edge tags and sorted, and the key store is released.  Nothing
// changes (the truncation stands) when the two layers and a minimal candidate buffer would not
// fit mem_cap.
int continue_sorted(cg_growth* h, cudaStream_t st, int* final_status) {
    const JobDev J = h->host_job;
    const int r = J.radius;
    if (r < 0 || J.hi < J.lo) return CG_EDEVICE;
    const uint64_t Fcur = J.hi - J.lo;
    std::vector<uint64_t> sizes((size_t)r + 1);
    cudaError_t e = cudaMemcpyAsync(sizes.data(), h->d_layers, sizeof(uint64_t) * sizes.size(),
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
    h->stats.d2h_bytes += sizeof(uint64_t) * sizes.size();
    const uint64_t Fprev = r > 0 ? sizes[r - 1] : 0;
    if (sizes[r] != Fcur || J.lo < Fprev) return CG_EDEVICE;
    const uint64_t mem = h->mem_cap ? h->mem_cap : kDefaultMemCap;
    // the first candidate buffer sorts the two layers; the steps size their own
    const uint64_t q0 = std::max<uint64_t>(std::max<uint64_t>(Fprev, Fcur), 4096);
    if (8 * (Fprev + Fcur) + cand_bytes(q0) > mem) return CG_OK;
    if (!h->d_count) {
        h->d_count = (unsigned long long*)dev_alloc(64, st);
        if (!h->d_count) return CG_ENOMEM;
    }
    dev_free(h->d_table, st);
    h->d_table = nullptr;
    h->table_slots = 0;
    const int cur = 0, prev = 1;
    int rc = ensure_layer(h, prev, std::max<uint64_t>(Fprev, 1), 0, st);
    if (rc == CG_OK) rc = ensure_layer(h, cur, std::max<uint64_t>(Fcur, 1), 0, st);
    if (rc) return rc;
    if (Fprev && (e = cudaMemcpyAsync(h->d_L[prev], h->d_keys + (J.lo - Fprev), Fprev * 8,
                                      cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(h->d_L[cur], h->d_keys + J.lo, Fcur * 8, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_rc(e);
    dev_free(h->d_keys, st);
    h->d_keys = nullptr;
    h->keys_cap = 0;
    h->last_layer_ptr = nullptr;
    h->last_layer_n = 0;
    if ((rc = ensure_cand(h, q0, st))) return rc;
    if (h->n * h->width <= 60) {
        if ((e = cg::launch_mask_keys(h->d_L[prev], Fprev, cg::kKeyBits60, st)) != cudaSuccess) return cuda_rc(e);
        if ((e = cg::launch_mask_keys(h->d_L[cur], Fcur, cg::kKeyBits60, st)) != cudaSuccess) return cuda_rc(e);
        h->stats.launches += 2;
    }
    const cg::SortScratch sc = cg::carve_sort_scratch(h->d_sort_scratch, h->cand_cap);
    const int bits = h->width * h->n;
    if ((e = cudaMemsetAsync(sc.err, 0, 4, st)) != cudaSuccess) return cuda_rc(e);
    const int lo = sort_low_bit(h);
    if ((e = cg::launch_radix_sort(h->d_L[prev], Fprev, bits, sc, st, lo)) != cudaSuccess) return cuda_rc(e);
    if ((e = cg::launch_radix_sort(h->d_L[cur], Fcur, bits, sc, st, lo)) != cudaSuccess) return cuda_rc(e);
    h->stats.launches += 2 * (1 + cg::sort_passes(bits, lo));
    h->sort_layers.assign(sizes.begin(), sizes.end());
    h->stats.switched_to_sort = 1;
    h->stats.sort_from = r;
    return sort_steps(h, st, cur, prev, Fcur, Fprev, r, final_status);
}

}  // namespace

extern "C" {

int cg_set_allocator(cg_alloc_fn alloc, cg_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return CG_EINVAL;
    g_alloc.alloc = alloc;
    g_alloc.free_fn = free_fn;
    g_alloc.ctx = ctx;
    return CG_OK;
}

int cg_growth_create(int n, int k, const uint8_t* gens, int inverse_closed, int max_radius,
                     uint64_t mem_cap, cg_growth_t* out) {
    if (out == nullptr) return CG_EINVAL;
    *out = nullptr;
    // n > 16: from the identity with 5-bit elements (n <= 25, two-word keys), or from a start
    // vector of narrow values (cg_growth_set_start), up to 128 elements
    int rc = validate(n, k, gens, cg::kMaxWideElems);
    if (rc) return rc;
    auto rows = clean_rows(n, k, gens);
    if (inverse_closed && !closed_under_inverse(rows, n)) return CG_ENOTCLOSED;
    cg_growth* h = new (std::nothrow) cg_growth();
    if (!h) return CG_ENOMEM;
    h->n = n;
    h->k = (int)rows.size();
    h->rows = rows;
    if (n <= cg::kMaxN) {
        h->gsm = make_gensms(rows, n);
    } else {
        h->width = 5;
        h->wide = true;
        if (n > 25 || !make_widegens(rows, n, 5, h->wgsm)) h->wgsm.clear();   // no growth from e
        for (int i = 0; i < n && n <= 25; ++i) {
            const int bit = 5 * i;
            if (bit < 64) h->wstart.lo |= (uint64_t)i << bit;
            if (bit + 5 > 64) h->wstart.hi |= bit >= 64 ? (uint64_t)i << (bit - 64) : (uint64_t)i >> (64 - bit);
        }
    }
    h->inverse_closed = inverse_closed ? 1 : 0;
    h->max_radius = max_radius < 0 ? -1 : max_radius;
    h->mem_cap = mem_cap ? mem_cap : kDefaultMemCap;
    std::vector<uint8_t> flat;
    for (auto& r : rows) flat.insert(flat.end(), r.begin(), r.end());
    h->order = rows.empty() ? 1 : cg::group_order(n, (int)rows.size(), flat.data());
    h->states_bound = h->order;
    *out = h;
    return CG_OK;
}

int cg_growth_set_start(cg_growth_t h, const uint8_t* start) {
    if (!h) return CG_EINVAL;
    int count[16] = {0};
    int maxv = 0;
    if (start)
        for (int i = 0; i < h->n; ++i) {
            if (start[i] > 15) return CG_EINVAL;
            count[start[i]]++;
            maxv = std::max(maxv, (int)start[i]);
        }
    // Permutations keep 4 bits per element (the rank-indexed strategies read them); other
    // vectors take the narrowest width that holds their values: binary vectors 1 bit.  Keys of
    // more than 64 bits, or generators that the one-word forms cannot express, take two words.
    bool distinct = true;
    for (int v = 0; v < 16; ++v) distinct &= count[v] <= 1;
    const bool is_perm = start && distinct && maxv < h->n;
    const int w = is_perm ? 4 : maxv <= 1 ? 1 : maxv <= 3 ? 2 : 4;
    if (start && h->n * w > 128) return CG_EINVAL;
    std::vector<GenSM> narrow;
    bool use_narrow = start && h->n * w <= 64;
    for (size_t j = 0; use_narrow && j < h->rows.size(); ++j) {
        GenSM G;
        use_narrow = make_gensm_checked(h->rows[j].data(), h->n, w, G);
    }
    std::vector<cg::WideGen> wg;
    if (start && !use_narrow && !make_widegens(h->rows, h->n, w, wg)) return CG_EINVAL;
    if (h->device >= 0) {                 // buffers were sized for the previous start
        h->release(nullptr);
        cudaStreamSynchronize(nullptr);
    }
    h->mode = -1;
    if (!start) {
        h->use_start = false;
        h->start_key = 0;
        h->start_is_perm = true;
        h->width = h->n <= cg::kMaxN ? 4 : 5;
        h->wide = h->n > cg::kMaxN;
        if (!h->wide) {
            h->gsm = make_gensms(h->rows, h->n, 4);
        } else if (h->n > 25 || !make_widegens(h->rows, h->n, 5, h->wgsm)) {
            h->wgsm.clear();
        }
        if (h->wide) {
            h->wstart = cg::Key128{0, 0};
            for (int i = 0; i < h->n && h->n <= 25; ++i) {
                const int bit = 5 * i;
                if (bit < 64) h->wstart.lo |= (uint64_t)i << bit;
                if (bit + 5 > 64) h->wstart.hi |= bit >= 64 ? (uint64_t)i << (bit - 64) : (uint64_t)i >> (64 - bit);
            }
        }
        h->states_bound = h->order;
        return CG_OK;
    }
    uint64_t key = 0;
    cg::Key128 wkey{0, 0};
    for (int i = 0; i < h->n; ++i) {
        const int bit = w * i;
        if (bit < 64) wkey.lo |= (uint64_t)start[i] << bit;
        else wkey.hi |= (uint64_t)start[i] << (bit - 64);
        if (bit < 64) key |= (uint64_t)start[i] << bit;
    }
    // The orbit of the start vector has at most as many states as the group, and at most as
    // many as the distinct rearrangements of the vector (a multinomial coefficient), computed as
    // a product of binomials, saturating at 2^64 - 1.
    uint64_t rearr = 1;
    int placed = 0;
    for (int v = 0; v < 16; ++v) {
        for (int j = 1; j <= count[v]; ++j) {   // rearr *= C(placed + j, j) / C(placed + j - 1, j - 1)
            ++placed;
            const unsigned __int128 x = (unsigned __int128)rearr * (unsigned)placed / (unsigned)j;
            rearr = x > (unsigned __int128)~0ull ? ~0ull : (uint64_t)x;
        }
    }
    h->use_start = true;
    h->start_key = key;
    h->start_constant = count[start[0]] == h->n;
    h->start_is_perm = is_perm;
    h->width = w;
    h->wide = !use_narrow;
    if (use_narrow) h->gsm = make_gensms(h->rows, h->n, w);
    else { h->wgsm = wg; h->gsm.clear(); }
    h->wstart = wkey;
    h->states_bound = std::min(h->order, rearr);
    return CG_OK;
}

int cg_growth_set_option(cg_growth_t h, int option, int64_t value) {
    if (!h) return CG_EINVAL;
    switch (option) {
        case CG_OPT_STRATEGY:
            if (value < CG_STRATEGY_AUTO || value > CG_STRATEGY_SWEEP) return CG_EINVAL;
            if (value == CG_STRATEGY_SORT && !h->inverse_closed) return CG_EINVAL;
            if (value != h->strategy && h->device >= 0) {   // buffers are laid out per strategy
                h->release(nullptr);
                cudaStreamSynchronize(nullptr);
            }
            h->mode = -1;
            h->strategy = (int)value;
            return CG_OK;
        case CG_OPT_STOP_ABOVE:
            if (value < 0) return CG_EINVAL;
            h->stop_above = (uint64_t)value;
            return CG_OK;
        case CG_OPT_KEEP_LAST:
            h->keep_last = value ? 1 : 0;
            return CG_OK;
        case CG_OPT_GRID:
            if (value < 0 || value > (1 << 20)) return CG_EINVAL;
            h->grid_override = (int)value;
            return CG_OK;
        case CG_OPT_ILP:
            if (value < 0 || value > 12 || (value > 4 && value < 9)) return CG_EINVAL;
            h->ilp_override = (int)value;
            return CG_OK;
        case CG_OPT_SWEEP_ORDER:
            if (value < cg::kSweepOrderAuto || value > cg::kSweepOrderRank) return CG_EINVAL;
            h->sweep_order = (int)value;
            return CG_OK;
        default:
            return CG_EINVAL;
    }
}

int cg_growth_run(cg_growth_t h, void* cuda_stream, uint64_t* layer_sizes_out, int cap,
                  int* num_layers_out) {
    if (!h || !layer_sizes_out || !num_layers_out || cap < 0) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    h->have_last = false;
    std::memset(&h->stats, 0, sizeof(h->stats));
    // from the identity beyond 16 elements: 5-bit elements in two words, n <= 25
    if (!h->use_start && h->wide && h->wgsm.empty()) return CG_EINVAL;
    // trivial group, radius 0, or a constant start vector (every permutation fixes it): one state
    if (h->k == 0 || h->max_radius == 0 || (h->use_start && h->start_constant)) {
        *num_layers_out = 1;
        if (cap < 1) return CG_EINVAL;
        layer_sizes_out[0] = 1;
        return (h->k == 0 || h->max_radius != 0) ? CG_OK : CG_TRUNC_RADIUS;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_rc(e);
    if (h->device >= 0 && h->device != dev) return CG_EINVAL;
    h->device = dev;
    int status = 0;
    if (h->wide) {
        int rc = run_wide(h, st, &status);
        if (rc) return rc;
        h->last_is_sweep = false;
        const int layers = h->host_job.radius + 1;
        *num_layers_out = layers;
        if (cap < layers) return CG_EINVAL;
        e = cudaMemcpyAsync(layer_sizes_out, h->d_layers, sizeof(uint64_t) * layers, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_rc(e);
        h->stats.d2h_bytes += sizeof(uint64_t) * layers;
        h->have_last = true;
        return status_to_rc(status);
    }
    const bool use_sort = h->strategy == CG_STRATEGY_SORT;
    const bool use_sweep = h->strategy == CG_STRATEGY_SWEEP ||
                           (h->strategy == CG_STRATEGY_AUTO && sweep_preferred(h));
    int rc = use_sort ? run_sort(h, st, &status)
                      : use_sweep ? run_sweep(h, st, &status) : run_hash(h, st, &status);
    if (rc) return rc;
    if (!use_sort && !use_sweep && status == cg::kNeedMem && h->strategy == CG_STRATEGY_AUTO &&
        h->inverse_closed) {
        if ((rc = continue_sorted(h, st, &status))) return rc;
    }
    const bool sorted = use_sort || h->stats.switched_to_sort;
    h->last_is_sweep = use_sweep;
    const int layers = h->host_job.radius + 1;
    *num_layers_out = layers;
    if (cap < layers) return CG_EINVAL;
    if (sorted) {
        for (int r = 0; r < layers; ++r) layer_sizes_out[r] = h->sort_layers[r];
    } else {
        e = cudaMemcpyAsync(layer_sizes_out, h->d_layers, sizeof(uint64_t) * layers,
                            cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
    h->stats.d2h_bytes += sizeof(uint64_t) * layers;
    h->have_last = true;
    return status_to_rc(status);
}

int cg_growth_last_layer(cg_growth_t h, uint64_t* keys_out, uint64_t cap, uint64_t* count_out) {
    if (!h || !count_out || !h->have_last) return CG_EINVAL;
    if (h->wide) {
        // two words a state (low, high), the parent-edge tags of stored states stripped
        const cg::WideDev& D = h->host_wide;
        const uint64_t cnt = D.hi - D.lo;
        *count_out = cnt;
        if (cap < cnt || (!keys_out && cnt > 0)) return CG_EINVAL;
        cudaError_t e = cudaMemcpy(keys_out, h->d_wkeys + D.lo, cnt * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && D.tagged)
            for (uint64_t i = 0; i < cnt; ++i) keys_out[2 * i + 1] &= (1ull << 60) - 1;
        return cuda_rc(e);
    }
    if (h->last_is_sweep) {
        // unrank the last layer's bitmap (layer R lives in F[R & 1], its blocks in L[R & 1])
        const SweepDev& D = h->host_sweep;
        uint64_t cnt = 0;
        cudaError_t e = cudaMemcpy(&cnt, h->d_layers + D.radius, 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_rc(e);
        *count_out = cnt;
        if (cap < cnt || (!keys_out && cnt > 0)) return CG_EINVAL;
        if (cnt == 0) return CG_OK;
        uint64_t* d_out = (uint64_t*)dev_alloc(cnt * 8 + 64, nullptr);
        if (!d_out) return CG_ENOMEM;
        unsigned long long* d_count = (unsigned long long*)(d_out + cnt);
        const int w = D.radius & 1;
        int grid = 0;
        cudaDeviceGetAttribute(&grid, cudaDevAttrMultiProcessorCount, h->device);
        e = cudaMemsetAsync(d_count, 0, 8, nullptr);
        if (e == cudaSuccess)
            e = cg::launch_sweep_export(D.F[w], D.L[w], D.lcount[w], h->n, d_out, cnt, d_count,
                                        std::max(grid, 1) * 8, nullptr);
        unsigned long long got = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&got, d_count, 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(keys_out, d_out, cnt * 8, cudaMemcpyDeviceToHost);
        dev_free(d_out, nullptr);
        cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) return cuda_rc(e);
        return got == cnt ? CG_OK : CG_EDEVICE;
    }
    const uint64_t cnt = h->last_layer_n;
    *count_out = cnt;
    if (cap < cnt || (!keys_out && cnt > 0)) return CG_EINVAL;
    cudaError_t e = cudaMemcpy(keys_out, h->last_layer_ptr, cnt * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h->n * h->width <= 60)   // strip the parent-edge tags of stored states
        for (uint64_t i = 0; i < cnt; ++i) keys_out[i] &= cg::kKeyBits60;
    return cuda_rc(e);
}

uint64_t cg_growth_group_order(cg_growth_t h) { return h ? h->order : 0; }

int cg_growth_key_width(cg_growth_t h) { return h ? h->width : 0; }

int cg_growth_key_words(cg_growth_t h) { return h ? (h->wide ? 2 : 1) : 0; }

const char* cg_last_error_detail(void) {
    if (g_last_cuda_error == cudaSuccess) return "";
    std::snprintf(g_last_detail, sizeof(g_last_detail), "%s at host_api.cu:%d",
                  cudaGetErrorName(g_last_cuda_error), g_last_cuda_line);
    return g_last_detail;
}

int cg_growth_get_stats(cg_growth_t h, cg_growth_stats* out) {
    if (!h || !out) return CG_EINVAL;
    *out = h->stats;
    return CG_OK;
}

int cg_growth_destroy(cg_growth_t h) {
    if (!h) return CG_OK;
    if (h->device >= 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur == h->device) {
            h->release(nullptr);
            cudaStreamSynchronize(nullptr);
            if (h->ev0) cudaEventDestroy(h->ev0);
            if (h->ev1) cudaEventDestroy(h->ev1);
        }
    }
    delete h;
    return CG_OK;
}

const char* cg_strerror(int code) {
    switch (code) {
        case CG_OK: return "ok: the growth ended (next layer empty)";
        case CG_TRUNC_RADIUS: return "stopped at max_radius (reported layers are exact)";
        case CG_TRUNC_MEMCAP: return "stopped: the next layer did not fit in mem_cap (reported layers are exact)";
        case CG_TRUNC_ABOVE: return "stopped after the first layer above stop_above (reported layers are exact)";
        case CG_EINVAL: return "invalid argument";
        case CG_ENOTCLOSED: return "generating set is not closed under inverse";
        case CG_ENOMEM: return "device memory allocation failed";
        case CG_ECUDA: return "CUDA runtime error";
        case CG_EDEVICE: return "kernel reported an internal error";
        case CG_ETIMEOUT: return "a bounded device-side wait timed out";
        case CG_ETOOBIG: return "problem exceeds the fixed scratch of cg_growth_run_noalloc";
        default: return "unknown code";
    }
}

// ---- step-level kernels ---------------------------------------------------------------------

int cg_expand(int n, int k, const uint8_t* gens, const uint64_t* frontier, uint64_t F,
              uint64_t* out, void* cuda_stream) {
    int rc = validate(n, k, gens);
    if (rc) return rc;
    if (F > 0 && (!frontier || !out)) return CG_EINVAL;
    if (F == 0) return CG_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<GenSM> g;
    for (int j = 0; j < k; ++j) g.push_back(make_gensm(gens + (size_t)j * n, n));
    GenSM* d = (GenSM*)dev_alloc(sizeof(GenSM) * k, st);
    if (!d) return CG_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(d, g.data(), sizeof(GenSM) * k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cg::launch_expand(d, k, frontier, F, out, 152 * 8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // g is host stack memory
    dev_free(d, st);
    return cuda_rc(e);
}

size_t cg_sort_unique_scratch_bytes(uint64_t n) { return cg::sort_scratch_bytes(n); }

int cg_sort_unique(uint64_t* keys, uint64_t n, int key_bits, uint64_t* out, uint64_t* d_count,
                   void* scratch, size_t scratch_bytes, void* cuda_stream) {
    if (key_bits < 1 || key_bits > 64 || !d_count) return CG_EINVAL;
    if (n > 0 && (!keys || !out || !scratch)) return CG_EINVAL;
    if (n > 0 && scratch_bytes < cg::sort_scratch_bytes(n)) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (n == 0) return cuda_rc(cudaMemsetAsync(d_count, 0, 8, st));
    cg::SortScratch sc = cg::carve_sort_scratch(scratch, n);
    cudaError_t e = cudaMemsetAsync(sc.err, 0, 4, st);
    if (e == cudaSuccess) e = cg::launch_radix_sort(keys, n, key_bits, sc, st);
    if (e == cudaSuccess)
        e = cg::launch_unique_difference(keys, n, nullptr, nullptr, 0, out,
                                         (unsigned long long*)d_count, sc, st);
    return cuda_rc(e);
}

int cg_set_difference(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb,
                      const uint64_t* c, uint64_t nc, uint64_t* out, uint64_t* d_count,
                      void* scratch, size_t scratch_bytes, void* cuda_stream) {
    if (!d_count) return CG_EINVAL;
    if ((na > 0 && (!a || !out || !scratch)) || (nb > 0 && !b) || (nc > 0 && !c)) return CG_EINVAL;
    if (na > 0 && scratch_bytes < cg::sort_scratch_bytes(na)) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (na == 0) return cuda_rc(cudaMemsetAsync(d_count, 0, 8, st));
    cg::SortScratch sc = cg::carve_sort_scratch(scratch, na);
    const uint64_t* bs[2] = {b, c};
    const unsigned long long ns[2] = {nb, nc};
    cudaError_t e = cudaMemsetAsync(sc.err, 0, 4, st);
    if (e == cudaSuccess)
        e = cg::launch_unique_difference(a, na, bs, ns, 2, out, (unsigned long long*)d_count, sc, st);
    return cuda_rc(e);
}

int cg_perm_rank(int n, const uint64_t* keys, uint64_t count, uint64_t* ranks, void* cuda_stream) {
    if (n < 1 || n > 16 || (count > 0 && (!keys || !ranks))) return CG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CG_ECUDA;
    return cuda_rc(cg::launch_pos_rank(keys, count, n, ranks, sms * 8, (cudaStream_t)cuda_stream));
}

int cg_perm_unrank(int n, const uint64_t* ranks, uint64_t count, uint64_t* keys, void* cuda_stream) {
    if (n < 1 || n > 16 || (count > 0 && (!keys || !ranks))) return CG_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CG_ECUDA;
    return cuda_rc(cg::launch_pos_unrank(ranks, count, n, keys, sms * 8, (cudaStream_t)cuda_stream));
}

int cg_shard_owner(uint64_t key, int P) {
    if (P < 1) return CG_EINVAL;
    return (int)(cg::mix64(key) % (uint64_t)P);
}

int cg_shard_expand(int n, int k, const uint8_t* gens, const uint64_t* frontier, uint64_t F, int P,
                    uint64_t* out, uint64_t cap, uint64_t* counts_out, void* cuda_stream) {
    int rc = validate(n, k, gens);
    if (rc) return rc;
    if (P < 1 || P > 4096 || !counts_out || (F > 0 && (!frontier || !out))) return CG_EINVAL;
    if (cap < (uint64_t)k * F) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<GenSM> g;
    for (int j = 0; j < k; ++j) g.push_back(make_gensm(gens + (size_t)j * n, n));
    const size_t gbytes = al_up(sizeof(GenSM) * k);
    char* d = (char*)dev_alloc(gbytes + 2 * sizeof(unsigned long long) * P + 256, st);
    if (!d) return CG_ENOMEM;
    GenSM* d_gens = reinterpret_cast<GenSM*>(d);
    unsigned long long* d_counts = reinterpret_cast<unsigned long long*>(d + gbytes);
    unsigned long long* d_cursor = d_counts + P;
    int* d_err = reinterpret_cast<int*>(d_cursor + P);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_gens, g.data(), sizeof(GenSM) * k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = cg::launch_owner_partition(d_gens, k, frontier, F, P, d_counts, d_cursor, out, cap, d_err,
                                       std::max(sms, 1) * 8, st);
    int derr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts_out, d_counts, sizeof(uint64_t) * P, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&derr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // g and derr live on the host stack
    dev_free(d, st);
    if (e != cudaSuccess) return cuda_rc(e);
    return derr ? derr : CG_OK;
}

int cg_hash_clear(uint64_t* table, uint64_t slots, void* cuda_stream) {
    if (!table && slots) return CG_EINVAL;
    return cuda_rc(cudaMemsetAsync(table, 0xFF, slots * 8, (cudaStream_t)cuda_stream));
}

int cg_hash_insert(uint64_t* table, uint64_t slots, const uint64_t* keys, uint64_t N,
                   uint64_t* new_out, uint64_t* new_count, void* cuda_stream) {
    if (!table || !new_count || slots == 0 || (slots & (slots - 1))) return CG_EINVAL;
    if (N > 0 && (!keys || !new_out)) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int* fail = (int*)dev_alloc(sizeof(int), st);
    if (!fail) return CG_ENOMEM;
    cudaError_t e = cudaMemsetAsync(fail, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(new_count, 0, sizeof(uint64_t), st);
    if (e == cudaSuccess && N > 0)
        e = cg::launch_hash_insert(table, slots - 1, keys, N, new_out,
                                   (unsigned long long*)new_count, fail, 152 * 8, st);
    dev_free(fail, st);
    return cuda_rc(e);
}

}  // extern "C"

// ---- batch of independent jobs ----------------------------------------------------------------
// The jobs are planned into launches ("waves") once: visited-set kind per job, waves within the
// memory budget and the L2 cap, one device buffer per wave with the jobs' static descriptors
// uploaded.  When all waves fit the budget together the buffers stay allocated between runs and
// a run is a fixed sequence per wave -- clear the visited sets, initialise the jobs, one
// persistent launch, copy the results to pinned host memory -- which CG_OPT_GRAPH captures once
// as a CUDA graph and replays.
struct cg_batch {
    struct Job {
        int n = 0, k = 0, max_radius = -1;
        std::vector<GenSM> gsm;
        uint64_t order = 1;
        uint64_t cap = 1;          // states the job may store
        int mode = cg::kVisitHash; // rank bitmap for small dense groups, else hash table
    };
    struct Wave {
        std::vector<int> ids;
        bool admit = false;        // one launch admitting its jobs by the L2 window (AdmitDev)
        char* base = nullptr;      // resident plans: the wave's device buffer
        uint64_t bytes = 0;
        uint64_t o_gens = 0, o_jobs = 0, o_ubeg = 0, o_ctl = 0, o_lay = 0, o_keys = 0, o_tab = 0;
        uint64_t o_adm = 0, o_act = 0, o_vis = 0;
        std::vector<uint64_t> vis;               // admit: visited bytes counted per job
        uint64_t window = 0;
        int max_active = 0;
        int unit_mult = 1;
        std::vector<uint64_t> slots;             // visited-set 8-byte slots per job
        std::vector<std::pair<uint64_t, uint64_t>> clear_runs[2];  // (offset, bytes): 0 -> 0x00, 1 -> 0xFF
        std::vector<GenSM> hg;
        std::vector<JobDev> hj;
        uint64_t h_off = 0;        // this wave's results in the pinned host buffer
    };
    std::vector<Job> jobs;
    uint64_t mem_cap = kDefaultMemCap;
    uint64_t wave_l2 = 0;          // cap on summed visited-set bytes per launch; 0: L2 / 2
    int ilp_override = 0;          // CG_OPT_ILP
    int grid_override = 0;         // CG_OPT_GRID
    int visited = 0;               // CG_OPT_BATCH_VISITED
    int use_graph = 1;             // CG_OPT_GRAPH (-1 after a failed capture)
    int max_active = 0;            // CG_OPT_BATCH_ACTIVE (0: min(jobs, 2048))
    int unit_mult = 4;             // CG_OPT_UNIT
    cg_growth_stats stats{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // the plan, rebuilt when an option or the layer capacity changes
    bool planned = false;
    int plan_cap = 0;
    int ilp = 1, grid = 0, device = -1;
    bool resident = false;
    std::vector<Wave> waves;
    char* h_pinned = nullptr;
    uint64_t h_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;  // stream the graph was captured on

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        gexec = nullptr;
        graph = nullptr;
    }
    void release() {
        drop_graph();
        for (auto& w : waves)
            if (w.base) dev_free(w.base, nullptr);
        waves.clear();
        if (h_pinned) cudaFreeHost(h_pinned);
        h_pinned = nullptr;
        h_bytes = 0;
        planned = false;
        resident = false;
        cudaStreamSynchronize(nullptr);
    }
};

namespace {

uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

// Lay out one wave's buffer: gens | jobs | ubeg | ctl | layers | keys | tables.
void layout_wave(cg_batch* b, cg_batch::Wave& w, int lcap) {
    const int nj = (int)w.ids.size();
    uint64_t ngens = 0, nkeys = 0, nslots = 0;
    std::vector<uint64_t> goff(nj), koff(nj), toff(nj);
    w.slots.assign(nj, 0);
    for (int i = 0; i < nj; ++i) {
        const auto& J = b->jobs[w.ids[i]];
        goff[i] = ngens; ngens += J.gsm.size();
        koff[i] = nkeys; nkeys += J.cap;
        w.slots[i] = J.mode == cg::kVisitBitmap ? bitmap_words(J.n) / 2 : table_slots_for(J.cap);
        toff[i] = nslots; nslots += w.slots[i];
    }
    w.o_gens = 0;
    w.o_jobs = al256(w.o_gens + ngens * sizeof(GenSM));
    w.o_ubeg = al256(w.o_jobs + nj * sizeof(JobDev));
    w.o_ctl = al256(w.o_ubeg + (nj + 1) * 8);
    w.o_lay = al256(w.o_ctl + sizeof(Ctl));
    w.o_keys = al256(w.o_lay + (uint64_t)nj * lcap * 8);
    w.o_tab = al256(w.o_keys + nkeys * 8);
    w.bytes = al256(w.o_tab + nslots * 8);
    if (w.admit) {
        w.o_adm = w.bytes;
        w.o_act = al256(w.o_adm + sizeof(cg::AdmitDev));
        w.o_vis = al256(w.o_act + 2ull * (uint64_t)w.max_active * sizeof(int));
        w.bytes = al256(w.o_vis + (uint64_t)nj * 8);
    }
    // visited sets: bitmaps start all-zero, hash tables all-ones; runs of one kind, one memset each
    for (auto& r : w.clear_runs) r.clear();
    for (int i = 0; i < nj;) {
        const int mode = b->jobs[w.ids[i]].mode;
        int j = i;
        uint64_t cnt = 0;
        while (j < nj && b->jobs[w.ids[j]].mode == mode) cnt += w.slots[j++];
        w.clear_runs[mode == cg::kVisitBitmap ? 0 : 1].push_back({w.o_tab + toff[i] * 8, cnt * 8});
        i = j;
    }
    // static descriptors (pointers filled in by bind_wave)
    w.hg.clear();
    w.hg.reserve(ngens);
    w.hj.assign(nj, JobDev{});
    for (int i = 0; i < nj; ++i) {
        const auto& J = b->jobs[w.ids[i]];
        w.hg.insert(w.hg.end(), J.gsm.begin(), J.gsm.end());
        JobDev& D = w.hj[i];
        std::memset(&D, 0, sizeof(D));
        D.keys = reinterpret_cast<uint64_t*>(koff[i] * 8);       // offsets until bound
        D.keys_cap = J.cap;
        D.table = reinterpret_cast<uint64_t*>(toff[i] * 8);
        D.table_mask = w.slots[i] - 1;
        D.gens = reinterpret_cast<const GenSM*>(goff[i] * sizeof(GenSM));
        D.layer_sizes = reinterpret_cast<uint64_t*>((uint64_t)i * lcap * 8);
        D.k = J.k;
        D.n = J.n;
        D.layers_cap = lcap;
        D.max_radius = J.max_radius;
        D.mode = J.mode;
        D.bitmap_words = J.mode == cg::kVisitBitmap ? bitmap_words(J.n) : 0;
        D.tagged = J.n <= 15 ? 1 : 0;
    }
}

// Turn the offsets of the wave's descriptors into device addresses of `base` and upload the
// static part (generators and descriptors).
cudaError_t bind_wave(cg_batch::Wave& w, char* base, cudaStream_t st) {
    std::vector<JobDev> hj = w.hj;
    for (auto& D : hj) {
        D.keys = reinterpret_cast<uint64_t*>(base + w.o_keys + reinterpret_cast<uint64_t>(D.keys));
        D.table = reinterpret_cast<uint64_t*>(base + w.o_tab + reinterpret_cast<uint64_t>(D.table));
        D.gens = reinterpret_cast<const GenSM*>(base + w.o_gens + reinterpret_cast<uint64_t>(D.gens));
        D.layer_sizes = reinterpret_cast<uint64_t*>(base + w.o_lay + reinterpret_cast<uint64_t>(D.layer_sizes));
    }
    cudaError_t e = cudaSuccess;
    if (!w.hg.empty()) e = cudaMemcpyAsync(base + w.o_gens, w.hg.data(), w.hg.size() * sizeof(GenSM),
                                           cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + w.o_jobs, hj.data(), hj.size() * sizeof(JobDev), cudaMemcpyHostToDevice, st);
    cg::AdmitDev A{};
    if (w.admit) {
        A.act[0] = reinterpret_cast<int*>(base + w.o_act);
        A.act[1] = A.act[0] + w.max_active;
        A.vis = reinterpret_cast<const uint64_t*>(base + w.o_vis);
        A.window = w.window;
        A.max_active = w.max_active;
        A.njobs = (int)w.ids.size();
        A.unit_mult = w.unit_mult;
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + w.o_adm, &A, sizeof(A), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + w.o_vis, w.vis.data(), w.vis.size() * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // hj, A are local copies
    return e;
}

// Results of one wave in host memory: descriptors, control block, layer sizes.
uint64_t wave_result_bytes(const cg_batch::Wave& w, int lcap) {
    return al256(w.ids.size() * sizeof(JobDev)) + al256(sizeof(Ctl)) + (uint64_t)w.ids.size() * lcap * 8;
}

// Enqueue one run of a bound wave: clear, initialise, grow, copy results to host memory `hout`.
cudaError_t enqueue_wave(cg_batch* b, cg_batch::Wave& w, char* base, char* hout, int lcap, cudaStream_t st) {
    const int nj = (int)w.ids.size();
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 2 && e == cudaSuccess; ++v)
        for (auto& r : w.clear_runs[v]) {
            e = cudaMemsetAsync(base + r.first, v ? 0xFF : 0, r.second, st);
            if (e != cudaSuccess) break;
        }
    JobDev* d_jobs = reinterpret_cast<JobDev*>(base + w.o_jobs);
    unsigned long long* d_ubeg = reinterpret_cast<unsigned long long*>(base + w.o_ubeg);
    Ctl* d_ctl = reinterpret_cast<Ctl*>(base + w.o_ctl);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctl, 0, sizeof(Ctl), st);
    if (w.admit) {
        // one launch for the whole batch: jobs are admitted (and set up) as the window allows
        const cg::AdmitDev* d_adm = reinterpret_cast<const cg::AdmitDev*>(base + w.o_adm);
        if (e == cudaSuccess) e = cg::launch_admit_first(d_jobs, d_ubeg, d_ctl, d_adm, st);
        if (e == cudaSuccess)
            e = cg::launch_hash_grow(d_jobs, nj, d_ubeg, d_ctl, b->grid, 1 << 30, kTimeoutNs, b->ilp, st,
                                     0, d_adm);
    } else {
        if (e == cudaSuccess) e = cg::launch_init_jobs(d_jobs, nj, d_ubeg, d_ctl, st);
        if (e == cudaSuccess)
            e = cg::launch_hash_grow(d_jobs, nj, d_ubeg, d_ctl, b->grid, lcap + 1, kTimeoutNs, b->ilp, st);
    }
    const uint64_t o1 = al256(nj * sizeof(JobDev)), o2 = o1 + al256(sizeof(Ctl));
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout, d_jobs, nj * sizeof(JobDev), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hout + o1, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hout + o2, base + w.o_lay, (uint64_t)nj * lcap * 8, cudaMemcpyDeviceToHost, st);
    return e;
}

// Read one wave's results from host memory into the caller's arrays.
int collect_wave(cg_batch* b, const cg_batch::Wave& w, const char* hres, int lcap, int cap,
                 uint64_t* layer_out, int* nl_out, int* status_out) {
    const int nj = (int)w.ids.size();
    const JobDev* hj = reinterpret_cast<const JobDev*>(hres);
    const uint64_t o1 = al256(nj * sizeof(JobDev)), o2 = o1 + al256(sizeof(Ctl));
    const Ctl* ctl = reinterpret_cast<const Ctl*>(hres + o1);
    const uint64_t* lay = reinterpret_cast<const uint64_t*>(hres + o2);
    b->stats.rounds += ctl->rounds;
    if (ctl->err) return ctl->err;
    int rc = CG_OK;
    for (int i = 0; i < nj; ++i) {
        const int j = w.ids[i];
        const int layers = hj[i].radius + 1;
        int st_rc = status_to_rc(hj[i].status);
        if (layers > cap) { st_rc = CG_EINVAL; rc = CG_EINVAL; }
        nl_out[j] = layers;
        for (int r = 0; r < layers && r < cap; ++r) layer_out[(uint64_t)j * cap + r] = lay[(uint64_t)i * lcap + r];
        if (status_out) status_out[j] = st_rc;
        if (st_rc < 0 && rc == CG_OK) rc = st_rc;
    }
    return rc;
}

// Choose visited sets, kernel variant, grid and waves; allocate the waves' buffers when they
// fit together.
int plan_batch(cg_batch* b, int dev, int cap, cudaStream_t st) {
    b->release();
    int maxk = 1;
    bool any_bitmap = false;
    for (auto& J : b->jobs) {
        maxk = std::max(maxk, J.k);
        const bool can_bitmap = J.k > 0 && J.n <= 12 && bitmap_fits(J.n, b->mem_cap);
        J.mode = (b->visited == CG_STRATEGY_HASH) ? cg::kVisitHash
                 : (b->visited == CG_STRATEGY_BITMAP) ? (can_bitmap ? cg::kVisitBitmap : cg::kVisitHash)
                 : (can_bitmap && bitmap_eligible(J.n, J.order, b->mem_cap)) ? cg::kVisitBitmap
                                                                              : cg::kVisitHash;
        any_bitmap |= J.mode == cg::kVisitBitmap;
    }
    // The rank-bitmap kernel variant also runs hash-table jobs of the same launch.
    const int base_ilp = b->ilp_override > 0 ? b->ilp_override : default_ilp(maxk, any_bitmap);
    b->ilp = base_ilp + (any_bitmap ? 16 : 0);
    b->stats.strategy_used = any_bitmap ? CG_STRATEGY_BITMAP : CG_STRATEGY_HASH;
    b->stats.probe_variant = b->ilp;
    const int grid_max = grow_grid(dev, b->ilp, true);
    if (grid_max <= 0) return CG_ECUDA;
    b->grid = b->grid_override > 0 ? std::min(grid_max, b->grid_override) : grid_max;
    const uint64_t budget = b->mem_cap;
    const uint64_t per_job_max = max_cap_for_mem(budget / 2);
    uint64_t l2_cap = b->wave_l2;
    if (l2_cap == 0) {
        int l2 = 0;
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) {
            cudaGetLastError();
            l2 = 64 << 20;
        }
        l2_cap = (uint64_t)l2 / 2;
    }
    // When every job's buffers fit the budget together, the batch is one launch that admits
    // the jobs in order as the L2 window allows (AdmitDev).  Otherwise greedy waves in job
    // order, each within the memory budget and with visited sets that together fit the L2 cap,
    // allocated and run one after the other.  Either way a set larger than the cap misses L2
    // wherever it runs and does not count.  Jobs with no work (no generator, radius 0) are
    // answered on the host.
    const int lcap = cap + 1;
    std::vector<uint64_t> need_of(b->jobs.size(), 0), vis_of(b->jobs.size(), 0);
    uint64_t all_need = 0;
    int with_work = 0;
    for (int j = 0; j < (int)b->jobs.size(); ++j) {
        auto& J = b->jobs[j];
        if (J.k == 0 || J.max_radius == 0) continue;
        J.cap = std::max<uint64_t>(1, std::min<uint64_t>(J.order, per_job_max));
        const uint64_t set_bytes = J.mode == cg::kVisitBitmap ? bitmap_words(J.n) * 4
                                                               : table_slots_for(J.cap) * 8;
        need_of[j] = J.cap * 8 + set_bytes + sizeof(GenSM) * J.gsm.size() + sizeof(JobDev) +
                     (uint64_t)lcap * 8 + 1024;
        vis_of[j] = set_bytes <= l2_cap ? set_bytes : 0;
        all_need += need_of[j] + 16;
        ++with_work;
    }
    uint64_t total_bytes = 0;
    if (with_work > 0 && all_need + (4ull << 20) <= budget) {
        cg_batch::Wave w;
        w.admit = true;
        w.window = l2_cap;
        w.max_active = b->max_active > 0 ? std::min(b->max_active, with_work) : std::min(with_work, 2048);
        w.unit_mult = b->unit_mult;
        for (int j = 0; j < (int)b->jobs.size(); ++j)
            if (need_of[j]) {
                w.ids.push_back(j);
                w.vis.push_back(vis_of[j]);
            }
        layout_wave(b, w, lcap);
        total_bytes = w.bytes;
        b->waves.push_back(std::move(w));
    } else {
        cg_batch::Wave cur;
        uint64_t wave_bytes = 0, wave_vis = 0;
        auto close_wave = [&]() {
            if (cur.ids.empty()) return;
            layout_wave(b, cur, lcap);
            total_bytes += cur.bytes;
            b->waves.push_back(std::move(cur));
            cur = cg_batch::Wave();
            wave_bytes = wave_vis = 0;
        };
        for (int j = 0; j < (int)b->jobs.size(); ++j) {
            if (!need_of[j]) continue;
            if (!cur.ids.empty() && (wave_bytes + need_of[j] > budget || wave_vis + vis_of[j] > l2_cap))
                close_wave();
            cur.ids.push_back(j);
            wave_bytes += need_of[j];
            wave_vis += vis_of[j];
        }
        close_wave();
    }
    // pinned host memory for every wave's results
    uint64_t hb = 0;
    for (auto& w : b->waves) {
        w.h_off = hb;
        hb += al256(wave_result_bytes(w, lcap));
    }
    if (hb) {
        if (cudaMallocHost(reinterpret_cast<void**>(&b->h_pinned), hb) != cudaSuccess) {
            cudaGetLastError();
            return CG_ENOMEM;
        }
        b->h_bytes = hb;
    }
    // resident when all waves fit the budget together
    b->resident = total_bytes <= budget;
    if (b->resident) {
        for (auto& w : b->waves) {
            w.base = (char*)dev_alloc(w.bytes, st);
            if (!w.base) { b->release(); return CG_ENOMEM; }
            cudaError_t e = bind_wave(w, w.base, st);
            if (e != cudaSuccess) { b->release(); return cuda_rc(e); }
            b->stats.h2d_bytes += w.hg.size() * sizeof(GenSM) + w.hj.size() * sizeof(JobDev);
        }
    }
    b->planned = true;
    b->plan_cap = cap;
    b->device = dev;
    return CG_OK;
}

// Enqueue a whole run of a resident plan (every wave).
cudaError_t enqueue_resident_run(cg_batch* b, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const int lcap = b->plan_cap + 1;
    for (auto& w : b->waves) {
        if (e != cudaSuccess) break;
        e = enqueue_wave(b, w, w.base, b->h_pinned + w.h_off, lcap, st);
    }
    return e;
}

}  // namespace

extern "C" {

int cg_batch_create(int njobs, const int* n, const int* k, const uint8_t* gens,
                    const uint64_t* gens_offset, const int* inverse_closed,
                    const int* max_radius, uint64_t mem_cap, cg_batch_t* out) {
    if (!out || njobs < 0 || (njobs > 0 && (!n || !k || !gens || !gens_offset))) return CG_EINVAL;
    *out = nullptr;
    cg_batch* b = new (std::nothrow) cg_batch();
    if (!b) return CG_ENOMEM;
    b->mem_cap = mem_cap ? mem_cap : kDefaultMemCap;
    b->jobs.resize(njobs);
    for (int j = 0; j < njobs; ++j) {
        const uint8_t* g = gens + gens_offset[j];
        int rc = validate(n[j], k[j], g);
        if (rc) { delete b; return rc; }
        auto rows = clean_rows(n[j], k[j], g);
        if (inverse_closed && inverse_closed[j] && !closed_under_inverse(rows, n[j])) {
            delete b;
            return CG_ENOTCLOSED;
        }
        auto& J = b->jobs[j];
        J.n = n[j];
        J.k = (int)rows.size();
        J.max_radius = (max_radius && max_radius[j] >= 0) ? max_radius[j] : -1;
        J.gsm = make_gensms(rows, n[j]);
        std::vector<uint8_t> flat;
        for (auto& r : rows) flat.insert(flat.end(), r.begin(), r.end());
        J.order = rows.empty() ? 1 : cg::group_order(n[j], (int)rows.size(), flat.data());
    }
    *out = b;
    return CG_OK;
}

int cg_batch_run(cg_batch_t b, void* cuda_stream, uint64_t* layer_sizes_out, int cap,
                 int* num_layers_out, int* status_out) {
    if (!b || !num_layers_out || cap < 1 || (!layer_sizes_out && !b->jobs.empty())) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::memset(&b->stats, 0, sizeof(b->stats));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_rc(e);
    if (!b->ev0 && (e = cudaEventCreate(&b->ev0)) != cudaSuccess) return cuda_rc(e);
    if (!b->ev1 && (e = cudaEventCreate(&b->ev1)) != cudaSuccess) return cuda_rc(e);
    // jobs with no work
    for (int j = 0; j < (int)b->jobs.size(); ++j) {
        const auto& J = b->jobs[j];
        if (J.k == 0 || J.max_radius == 0) {
            num_layers_out[j] = 1;
            layer_sizes_out[(uint64_t)j * cap] = 1;
            if (status_out) status_out[j] = J.k == 0 ? CG_OK : CG_TRUNC_RADIUS;
        }
    }
    int rc = CG_OK;
    if (!b->planned || b->plan_cap != cap || b->device != dev) {
        if ((rc = plan_batch(b, dev, cap, st)) != CG_OK) return rc;
    } else {
        b->stats.strategy_used = b->ilp >= 16 ? CG_STRATEGY_BITMAP : CG_STRATEGY_HASH;
        b->stats.probe_variant = b->ilp;
    }
    const int lcap = cap + 1;
    if (b->resident) {
        if (b->use_graph > 0 && !b->gexec) {
            // capture the run once (a legacy-default stream cannot be captured: use our own)
            if (!b->gstream && cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                b->use_graph = -1;
            }
            if (b->use_graph > 0) {
                cudaStreamSynchronize(st);
                e = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t ee = enqueue_resident_run(b, b->gstream);
                    e = cudaStreamEndCapture(b->gstream, &b->graph);
                    if (ee != cudaSuccess) e = ee;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
                if (e != cudaSuccess) {         // capture not possible here: run without a graph
                    cudaGetLastError();
                    b->drop_graph();
                    b->use_graph = -1;
                }
            }
        }
        if (b->gexec) {
            // the replay starts after the caller's stream's earlier work (ev0 recorded there)
            if ((e = cudaEventRecord(b->ev0, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaStreamWaitEvent(b->gstream, b->ev0, 0)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaGraphLaunch(b->gexec, b->gstream)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaEventRecord(b->ev1, b->gstream)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaStreamSynchronize(b->gstream)) != cudaSuccess) return cuda_rc(e);
            // one graph launch: its kernels are counted below
        } else {
            if ((e = cudaEventRecord(b->ev0, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = enqueue_resident_run(b, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaEventRecord(b->ev1, st)) != cudaSuccess) return cuda_rc(e);
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
        }
        b->stats.kernel_ms += elapsed_ms(b->ev0, b->ev1);
        for (auto& w : b->waves) {
            b->stats.launches += w.admit ? 2 : 3;     // (admit_first | init_jobs + init_units) + grow
            b->stats.d2h_bytes += wave_result_bytes(w, lcap);
            int r = collect_wave(b, w, b->h_pinned + w.h_off, lcap, cap, layer_sizes_out,
                                 num_layers_out, status_out);
            if (r != CG_OK && rc == CG_OK) rc = r;
        }
        return rc;
    }
    // Not resident: each wave's buffer is allocated, run and freed in turn.
    for (auto& w : b->waves) {
        char* base = (char*)dev_alloc(w.bytes, st);
        if (!base) return CG_ENOMEM;
        e = bind_wave(w, base, st);
        b->stats.h2d_bytes += w.hg.size() * sizeof(GenSM) + w.hj.size() * sizeof(JobDev);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev0, st);
        if (e == cudaSuccess) e = enqueue_wave(b, w, base, b->h_pinned + w.h_off, lcap, st);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev1, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) b->stats.kernel_ms += elapsed_ms(b->ev0, b->ev1);
        dev_free(base, st);
        cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_rc(e);
        b->stats.launches += 3;
        b->stats.d2h_bytes += wave_result_bytes(w, lcap);
        int r = collect_wave(b, w, b->h_pinned + w.h_off, lcap, cap, layer_sizes_out, num_layers_out,
                             status_out);
        if (r != CG_OK && rc == CG_OK) rc = r;
    }
    return rc;
}

int cg_batch_set_option(cg_batch_t b, int option, int64_t value) {
    if (!b) return CG_EINVAL;
    switch (option) {
        case CG_OPT_ILP:
            if (value < 0 || value > 4) return CG_EINVAL;
            b->ilp_override = (int)value;
            break;
        case CG_OPT_GRID:
            if (value < 0 || value > (1 << 20)) return CG_EINVAL;
            b->grid_override = (int)value;
            break;
        case CG_OPT_BATCH_WAVE_L2:
            b->wave_l2 = value < 0 ? ~0ull : (uint64_t)value;
            break;
        case CG_OPT_BATCH_VISITED:
            if (value != CG_STRATEGY_AUTO && value != CG_STRATEGY_HASH && value != CG_STRATEGY_BITMAP)
                return CG_EINVAL;
            b->visited = (int)value;
            break;
        case CG_OPT_GRAPH:
            b->use_graph = value ? 1 : 0;
            b->drop_graph();
            return CG_OK;
        case CG_OPT_BATCH_ACTIVE:
            if (value < 0 || value > (1 << 20)) return CG_EINVAL;
            b->max_active = (int)value;
            break;
        case CG_OPT_UNIT:
            if (value != 1 && value != 2 && value != 4 && value != 8) return CG_EINVAL;
            b->unit_mult = (int)value;
            break;
        default:
            return CG_EINVAL;
    }
    if (b->planned) b->release();
    return CG_OK;
}

int cg_batch_set_wave_l2(cg_batch_t b, uint64_t bytes) {
    return cg_batch_set_option(b, CG_OPT_BATCH_WAVE_L2, bytes == ~0ull ? -1 : (int64_t)bytes);
}

int cg_batch_get_stats(cg_batch_t b, cg_growth_stats* out) {
    if (!b || !out) return CG_EINVAL;
    *out = b->stats;
    return CG_OK;
}

int cg_batch_destroy(cg_batch_t b) {
    if (!b) return CG_OK;
    b->release();
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
    return CG_OK;
}

}  // extern "C"

// ---- serving: continuous batching of growth jobs ------------------------------------------------
// Jobs are queued on the host, admitted into device slots while their predicted memory fits the
// budget, and every cg_server_step runs up to `rounds_per_step` layer steps of every admitted
// job in one persistent launch.  A job's states and visited set stay on the device between
// steps; finished jobs release their slot and memory at the end of the step in which they end,
// and queued jobs take their place at the start of the next step.
#include <deque>
#include <unordered_map>

namespace {

constexpr int kSrvMaxGens = 128;     // generators per job
// A job predicted to reach at least this many states fills the GPU by itself: it is grown
// alone by the single-job kernels (the fastest for it) when it reaches the head of the queue,
// and the smaller jobs around it are batched.
constexpr uint64_t kSrvSoloStates = CG_SERVER_SOLO_STATES;
constexpr int kSrvLayers = 4096;     // layer sizes kept per job (more: CG_TRUNC_RADIUS)

// Upper bound on the states a job visits up to its radius cap: sphere r of a graph of
// out-degree k has at most k (k-1)^(r-1) elements when the set is inverse-closed (no walk
// returns along the edge it came by), k^r otherwise; never more than the group order.
uint64_t predict_states(int k, uint64_t order, int max_radius, bool inverse_closed) {
    if (max_radius < 0) return order;
    uint64_t total = 1, layer = 1;
    for (int r = 1; r <= max_radius; ++r) {
        const uint64_t f = (r == 1 || !inverse_closed) ? (uint64_t)k : (uint64_t)(k > 1 ? k - 1 : 1);
        layer = (layer > order / std::max<uint64_t>(f, 1)) ? order : layer * f;
        total += std::min(layer, order);
        if (total >= order) return order;
    }
    return std::min(total, order);
}

// Device memory plan of one served job: the predicted states up to its radius cap (`want`),
// and the states it may store within `share` bytes (`cap`) with the cheaper visited set -- a
// hash table (8-byte key + 16 bytes of table per state at load 0.5) or, for n <= 14, the rank
// bitmap (n!/8 bytes whatever the states).  A job whose prediction exceeds the share gets the
// share and stops with CG_TRUNC_MEMCAP if it really needs more.
struct SrvPlan {
    uint64_t want = 1, cap = 1, bytes = 0, visited_words = 0;
    int mode = cg::kVisitHash;
};

SrvPlan plan_server_job(int n, int k, uint64_t order, int max_radius, bool inverse_closed, uint64_t share) {
    SrvPlan P;
    P.want = std::max<uint64_t>(1, predict_states(std::max(k, 1), order, max_radius, inverse_closed));
    uint64_t hcap = P.want;
    if (bytes_for(hcap) > share) hcap = std::max<uint64_t>(1, max_cap_for_mem(share));
    uint64_t bcap = 0;
    const uint64_t bm_bytes = (n >= 2 && n <= 14) ? bitmap_words(n) * 4 : ~0ull;
    if (bm_bytes < share) bcap = std::min<uint64_t>(P.want, (share - bm_bytes) / 8);
    const uint64_t hbytes = hcap * 8 + table_slots_for(hcap) * 8;
    const bool bitmap = bcap > hcap || (bcap == hcap && bcap > 0 && bcap * 8 + bm_bytes <= hbytes);
    if (bitmap) {
        P.mode = cg::kVisitBitmap;
        P.cap = std::max<uint64_t>(bcap, 1);
        P.visited_words = bm_bytes / 8;
    } else {
        P.mode = cg::kVisitHash;
        P.cap = hcap;
        P.visited_words = table_slots_for(hcap);
    }
    P.bytes = ((P.cap * 8 + 255) & ~255ull) + P.visited_words * 8;
    return P;
}

}  // namespace

struct cg_server {
    struct Job {
        uint64_t id = 0;
        int n = 0, k = 0, max_radius = -1;
        std::vector<GenSM> gsm;
        uint64_t order = 1, cap = 1, bytes = 0, visited_words = 0;
        int mode = cg::kVisitHash;
        bool solo = false;                 // predicted to fill the GPU: grown alone
        int inverse_closed = 0;
        std::vector<uint8_t> rows;         // distinct rows, k * n bytes (for a solo growth)
    };
    struct Slot {
        bool used = false;
        Job job;
        char* mem = nullptr;
    };
    struct Result {
        std::vector<uint64_t> layers;
        int status = 0;
    };
    uint64_t budget = 0, used = 0, job_cap_bytes = 0;
    int max_slots = 0, rounds_per_step = 8, active = 0, device = -1;
    std::deque<Job> queue;
    std::vector<Slot> slots;
    std::vector<JobDev> h_jobs;
    std::unordered_map<uint64_t, Result> results;
    std::vector<uint64_t> finished;
    uint64_t next_id = 1;
    JobDev* d_jobs = nullptr;
    unsigned long long* d_ubeg = nullptr;
    Ctl* d_ctl = nullptr;
    GenSM* d_gens = nullptr;
    uint64_t* d_layers = nullptr;
};

namespace {

int server_init_device(cg_server* s, cudaStream_t st) {
    if (s->d_jobs) return CG_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_rc(e);
    s->device = dev;
    const int m = s->max_slots;
    s->d_jobs = (JobDev*)dev_alloc(sizeof(JobDev) * m, st);
    s->d_ubeg = (unsigned long long*)dev_alloc(8 * (m + 1), st);
    s->d_ctl = (Ctl*)dev_alloc(sizeof(Ctl), st);
    s->d_gens = (GenSM*)dev_alloc(sizeof(GenSM) * kSrvMaxGens * m, st);
    s->d_layers = (uint64_t*)dev_alloc(8ull * kSrvLayers * m, st);
    if (!s->d_jobs || !s->d_ubeg || !s->d_ctl || !s->d_gens || !s->d_layers) return CG_ENOMEM;
    s->h_jobs.assign(m, JobDev{});
    for (auto& J : s->h_jobs) {
        std::memset(&J, 0, sizeof(J));
        J.status = cg::kEmptySlot;
    }
    if ((e = cudaMemcpyAsync(s->d_jobs, s->h_jobs.data(), sizeof(JobDev) * m, cudaMemcpyHostToDevice, st)))
        return cuda_rc(e);
    return CG_OK;
}

// Move queued jobs into free slots while the budget allows (first come, first served).
int server_admit(cg_server* s, cudaStream_t st) {
    while (!s->queue.empty()) {
        int free_slot = -1;
        for (int i = 0; i < s->max_slots; ++i)
            if (!s->slots[i].used) { free_slot = i; break; }
        if (free_slot < 0) break;
        cg_server::Job& q = s->queue.front();
        if (q.solo) break;                      // grown alone by cg_server_step, in order
        if (s->used + q.bytes > s->budget && s->active > 0) break;
        char* mem = (char*)dev_alloc(q.bytes, st);
        if (!mem) {
            if (s->active > 0) break;    // wait for memory to free up
            return CG_ENOMEM;
        }
        cg_server::Slot& sl = s->slots[free_slot];
        sl.used = true;
        sl.job = q;
        sl.mem = mem;
        s->queue.pop_front();
        s->used += sl.job.bytes;
        s->active += 1;
        const cg_server::Job& J = sl.job;
        JobDev D;
        std::memset(&D, 0, sizeof(D));
        D.keys = reinterpret_cast<uint64_t*>(mem);
        D.keys_cap = J.cap;
        D.table = reinterpret_cast<uint64_t*>(mem + J.cap * 8);
        D.table_mask = J.mode == cg::kVisitBitmap ? 0 : J.visited_words - 1;
        D.gens = s->d_gens + (size_t)free_slot * kSrvMaxGens;
        D.layer_sizes = s->d_layers + (size_t)free_slot * kSrvLayers;
        D.k = J.k;
        D.n = J.n;
        D.layers_cap = kSrvLayers;
        D.max_radius = J.max_radius;
        D.mode = J.mode;
        D.bitmap_words = J.mode == cg::kVisitBitmap ? bitmap_words(J.n) : 0;
        D.tagged = J.n <= 15 ? 1 : 0;
        D.status = cg::kFresh;
        s->h_jobs[free_slot] = D;
        cudaError_t e;
        if ((e = cudaMemcpyAsync((void*)D.gens, J.gsm.data(), sizeof(GenSM) * J.k, cudaMemcpyHostToDevice, st)))
            return cuda_rc(e);
        if ((e = cudaMemsetAsync(D.table, J.mode == cg::kVisitBitmap ? 0 : 0xFF, J.visited_words * 8, st)))
            return cuda_rc(e);
        if ((e = cudaMemcpyAsync(s->d_jobs + free_slot, &s->h_jobs[free_slot], sizeof(JobDev),
                                 cudaMemcpyHostToDevice, st)))
            return cuda_rc(e);
    }
    return CG_OK;
}

// Grow the solo job at the head of the queue alone with the single-job path: the same visited
// set and per-job share the batched launch would give it (so the same layers), no hand-off to
// the sorted step.  Its result joins the finished list.
int server_run_solo(cg_server* s, cudaStream_t st) {
    cg_server::Job J = std::move(s->queue.front());
    s->queue.pop_front();
    cg_growth_t g = nullptr;
    // a served job keeps at most kSrvLayers layers, as in the batched launch
    const int rad = (J.max_radius < 0 || J.max_radius > kSrvLayers - 1) ? kSrvLayers - 1 : J.max_radius;
    int rc = cg_growth_create(J.n, J.k, J.rows.data(), J.inverse_closed, rad, s->job_cap_bytes, &g);
    if (rc) return rc;
    rc = cg_growth_set_option(g, CG_OPT_STRATEGY,
                              J.mode == cg::kVisitBitmap ? CG_STRATEGY_BITMAP : CG_STRATEGY_HASH);
    std::vector<uint64_t> layers(kSrvLayers);
    int nl = 0;
    if (rc == CG_OK) rc = cg_growth_run(g, st, layers.data(), kSrvLayers, &nl);
    cg_growth_destroy(g);
    if (rc < 0) return rc;
    cg_server::Result R;
    R.layers.assign(layers.begin(), layers.begin() + nl);
    R.status = rc;
    s->results[J.id] = std::move(R);
    s->finished.push_back(J.id);
    return CG_OK;
}

}  // namespace

extern "C" {

int cg_server_create(uint64_t mem_budget, int max_slots, uint64_t job_mem_cap, int rounds_per_step,
                     cg_server_t* out) {
    if (!out || max_slots < 1 || max_slots > 4096 || rounds_per_step < 1) return CG_EINVAL;
    *out = nullptr;
    cg_server* s = new (std::nothrow) cg_server();
    if (!s) return CG_ENOMEM;
    s->budget = mem_budget ? mem_budget : kDefaultMemCap;
    s->job_cap_bytes = job_mem_cap ? job_mem_cap : std::max<uint64_t>(s->budget / 64, 1ull << 20);
    s->max_slots = max_slots;
    s->rounds_per_step = rounds_per_step;
    s->slots.resize(max_slots);
    *out = s;
    return CG_OK;
}

int cg_server_submit(cg_server_t s, int n, int k, const uint8_t* gens, int inverse_closed,
                     int max_radius, uint64_t* job_id_out) {
    if (!s || !job_id_out) return CG_EINVAL;
    int rc = validate(n, k, gens);
    if (rc) return rc;
    auto rows = clean_rows(n, k, gens);
    if (inverse_closed && !closed_under_inverse(rows, n)) return CG_ENOTCLOSED;
    if ((int)rows.size() > kSrvMaxGens) return CG_EINVAL;
    cg_server::Job J;
    J.id = s->next_id++;
    J.n = n;
    J.k = (int)rows.size();
    J.max_radius = max_radius < 0 ? -1 : max_radius;
    J.gsm = make_gensms(rows, n);
    std::vector<uint8_t> flat;
    for (auto& r : rows) flat.insert(flat.end(), r.begin(), r.end());
    J.order = rows.empty() ? 1 : cg::group_order(n, (int)rows.size(), flat.data());
    // predicted memory: states up to the radius cap, within the per-job share
    const SrvPlan P = plan_server_job(n, J.k, J.order, J.max_radius, inverse_closed != 0, s->job_cap_bytes);
    J.mode = P.mode;
    J.visited_words = P.visited_words;
    J.cap = P.cap;
    J.bytes = P.bytes;
    J.solo = P.want >= kSrvSoloStates;
    J.inverse_closed = inverse_closed ? 1 : 0;
    J.rows = flat;
    if (J.k == 0 || J.max_radius == 0) {       // only the identity: done at once
        cg_server::Result R;
        R.layers = {1};
        R.status = J.k == 0 ? CG_OK : CG_TRUNC_RADIUS;
        s->results[J.id] = R;
        s->finished.push_back(J.id);
    } else {
        s->queue.push_back(std::move(J));
    }
    *job_id_out = s->next_id - 1;
    return CG_OK;
}

int cg_server_predict(int n, int k, const uint8_t* gens, int inverse_closed, int max_radius,
                      uint64_t job_mem_cap, uint64_t* states_out, uint64_t* granted_out,
                      uint64_t* bytes_out, int* visited_out) {
    int rc = validate(n, k, gens);
    if (rc) return rc;
    if (job_mem_cap == 0) return CG_EINVAL;
    auto rows = clean_rows(n, k, gens);
    if (inverse_closed && !closed_under_inverse(rows, n)) return CG_ENOTCLOSED;
    std::vector<uint8_t> flat;
    for (auto& r : rows) flat.insert(flat.end(), r.begin(), r.end());
    const uint64_t order = rows.empty() ? 1 : cg::group_order(n, (int)rows.size(), flat.data());
    const int rad = max_radius < 0 ? -1 : max_radius;
    const SrvPlan P = plan_server_job(n, (int)rows.size(), order, rad, inverse_closed != 0, job_mem_cap);
    if (states_out) *states_out = P.want;
    if (granted_out) *granted_out = P.cap;
    if (bytes_out) *bytes_out = P.bytes;
    if (visited_out) *visited_out = P.mode == cg::kVisitBitmap ? CG_STRATEGY_BITMAP : CG_STRATEGY_HASH;
    return CG_OK;
}

int cg_server_step(cg_server_t s, void* cuda_stream, int* active_out, int* finished_out) {
    if (!s) return CG_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = server_init_device(s, st);
    if (rc) return rc;
    const size_t finished_before = s->finished.size();
    if (!s->queue.empty() && s->queue.front().solo) {
        if ((rc = server_run_solo(s, st))) return rc;
    }
    if ((rc = server_admit(s, st))) return rc;
    if (s->active > 0) {
        int maxk = 1;
        bool any_bitmap = false;
        for (auto& sl : s->slots)
            if (sl.used) {
                maxk = std::max(maxk, sl.job.k);
                any_bitmap |= sl.job.mode == cg::kVisitBitmap;
            }
        const int variant = default_ilp(maxk, any_bitmap) + (any_bitmap ? 16 : 0);
        const int grid = grow_grid(s->device, variant, true);
        if (grid <= 0) return CG_ECUDA;
        cudaError_t e;
        if ((e = cudaMemsetAsync(s->d_ctl, 0, sizeof(Ctl), st))) return cuda_rc(e);
        if ((e = cg::launch_init_jobs(s->d_jobs, s->max_slots, s->d_ubeg, s->d_ctl, st, 1))) return cuda_rc(e);
        if ((e = cg::launch_hash_grow(s->d_jobs, s->max_slots, s->d_ubeg, s->d_ctl, grid,
                                      s->rounds_per_step, kTimeoutNs, variant, st)))
            return cuda_rc(e);
        Ctl ctl;
        if ((e = cudaMemcpyAsync(s->h_jobs.data(), s->d_jobs, sizeof(JobDev) * s->max_slots,
                                 cudaMemcpyDeviceToHost, st)))
            return cuda_rc(e);
        if ((e = cudaMemcpyAsync(&ctl, s->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st))) return cuda_rc(e);
        if ((e = cudaStreamSynchronize(st))) return cuda_rc(e);
        if (ctl.err) return ctl.err;
        // retire the jobs that ended in this step
        std::vector<int> ended;
        for (int i = 0; i < s->max_slots; ++i) {
            if (!s->slots[i].used) continue;
            const int stt = s->h_jobs[i].status;
            if (stt != cg::kRunning && stt != cg::kFresh) ended.push_back(i);
        }
        std::vector<std::vector<uint64_t>> lay(ended.size());
        for (size_t q = 0; q < ended.size(); ++q) {
            const int i = ended[q];
            lay[q].resize(s->h_jobs[i].radius + 1);
            if ((e = cudaMemcpyAsync(lay[q].data(), s->d_layers + (size_t)i * kSrvLayers,
                                     8 * lay[q].size(), cudaMemcpyDeviceToHost, st)))
                return cuda_rc(e);
        }
        if (!ended.empty() && (e = cudaStreamSynchronize(st))) return cuda_rc(e);
        for (size_t q = 0; q < ended.size(); ++q) {
            const int i = ended[q];
            cg_server::Slot& sl = s->slots[i];
            cg_server::Result R;
            R.layers = std::move(lay[q]);
            R.status = status_to_rc(s->h_jobs[i].status);
            s->results[sl.job.id] = std::move(R);
            s->finished.push_back(sl.job.id);
            dev_free(sl.mem, st);
            sl.mem = nullptr;
            sl.used = false;
            s->used -= sl.job.bytes;
            s->active -= 1;
            s->h_jobs[i].status = cg::kEmptySlot;
            if ((e = cudaMemcpyAsync(s->d_jobs + i, &s->h_jobs[i], sizeof(JobDev), cudaMemcpyHostToDevice, st)))
                return cuda_rc(e);
        }
        if (!ended.empty() && (e = cudaStreamSynchronize(st))) return cuda_rc(e);
    }
    if (active_out) *active_out = s->active;
    if (finished_out) *finished_out = (int)(s->finished.size() - finished_before);
    return CG_OK;
}

int cg_server_finished(cg_server_t s, uint64_t* ids_out, int cap, int* count_out) {
    if (!s || !count_out || cap < 0) return CG_EINVAL;
    const int n = (int)std::min<size_t>(s->finished.size(), (size_t)cap);
    for (int i = 0; i < n; ++i) ids_out[i] = s->finished[i];
    s->finished.erase(s->finished.begin(), s->finished.begin() + n);
    *count_out = n;
    return CG_OK;
}

int cg_server_result(cg_server_t s, uint64_t job_id, uint64_t* layers_out, int cap,
                     int* num_layers_out, int* status_out) {
    if (!s || !num_layers_out || !status_out) return CG_EINVAL;
    auto it = s->results.find(job_id);
    if (it == s->results.end()) {
        *num_layers_out = -1;
        return CG_EINVAL;
    }
    const int nl = (int)it->second.layers.size();
    *num_layers_out = nl;
    *status_out = it->second.status;
    if (cap < nl || !layers_out) return CG_EINVAL;
    for (int r = 0; r < nl; ++r) layers_out[r] = it->second.layers[r];
    s->results.erase(it);
    return CG_OK;
}

int cg_server_load(cg_server_t s, int* queued, int* active, uint64_t* used_bytes) {
    if (!s) return CG_EINVAL;
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = s->active;
    if (used_bytes) *used_bytes = s->used;
    return CG_OK;
}

int cg_server_destroy(cg_server_t s) {
    if (!s) return CG_OK;
    if (s->device >= 0) {
        for (auto& sl : s->slots) dev_free(sl.mem, nullptr);
        dev_free(s->d_jobs, nullptr);
        dev_free(s->d_ubeg, nullptr);
        dev_free(s->d_ctl, nullptr);
        dev_free(s->d_gens, nullptr);
        dev_free(s->d_layers, nullptr);
        cudaStreamSynchronize(nullptr);
    }
    delete s;
    return CG_OK;
}

}  // extern "C"
