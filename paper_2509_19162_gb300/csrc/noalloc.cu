// Growth of a small Cayley graph without any memory allocation.
//
// Some callers cannot allocate device memory at the point where they want a growth: code
// running inside a memory-capped sandbox or pre-reserved pool, a real-time or inference
// process that forbids cudaMalloc after start-up (it would synchronise the device and
// fragment a carefully sized heap), or a plugin whose host application owns every
// allocation.  cg_growth_run_noalloc serves them: every buffer it needs lives in one
// file-scope device array of fixed size, g_noalloc_scratch, created when the CUDA module
// is loaded and held by every GPU that loads the library until the process exits.
//
// The array is shared by all calls and keeps the previous call's contents; each call clears
// what must start empty (visited table, control block) itself.  Calls are serialised on the
// host by a mutex and each call waits for its own stream, so two calls never overlap; work a
// caller launches that touches this array concurrently (none of the library's other entry
// points do) would race with it.
#include <cstring>
#include <mutex>

#include "../../include/cg_growth.h"
#include "cg_internal.h"
#include "cg_kernels.h"

namespace {

constexpr uint64_t kMaxStates = CG_NOALLOC_MAX_STATES;          // states the growth may visit
constexpr uint64_t kTableSlots = 2 * kMaxStates;                // load factor <= 0.5
constexpr int kMaxGens = CG_NOALLOC_MAX_GENS;
constexpr uint64_t kTimeoutNs = 30ull * 1000 * 1000 * 1000;

// Layout of the scratch array (byte offsets, each 256-aligned).
constexpr uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }
constexpr uint64_t kOffKeys = 0;
constexpr uint64_t kOffTable = align256(kOffKeys + kMaxStates * 8);
constexpr uint64_t kOffLayers = align256(kOffTable + kTableSlots * 8);
constexpr uint64_t kOffGens = align256(kOffLayers + (uint64_t)cg::kMaxLayers * 8);
constexpr uint64_t kOffJob = align256(kOffGens + (uint64_t)kMaxGens * sizeof(cg::GenSM));
constexpr uint64_t kOffCtl = align256(kOffJob + sizeof(cg::JobDev));
constexpr uint64_t kOffUbeg = align256(kOffCtl + sizeof(cg::Ctl));
constexpr uint64_t kScratchBytes = align256(kOffUbeg + 2 * sizeof(unsigned long long));

}  // namespace

// The fixed scratch: 8 MiB of states, 16 MiB of visited table and ~0.2 MiB of control data.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char* g_scratch_addr[64] = {};   // device address of g_noalloc_scratch, per device
int g_grid[64][5] = {};                   // co-resident blocks per device and probe ILP 1..4

// Once per device, with that device current: the device address of the scratch array (the
// array's name in host code is only a host-side stand-in, not a device address).  The cached
// address does not survive cudaDeviceReset: a process that resets a device must not call this
// entry point on it again.
int setup_device(int dev) {
    if (dev < 0 || dev >= 64) return CG_EINVAL;
    if (g_scratch_addr[dev]) return CG_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return CG_ECUDA;
    }
    for (int ilp = 1; ilp <= 4; ++ilp) {
        const int grid = cg::hash_grow_max_grid(dev, ilp, false);
        if (grid <= 0) return CG_ECUDA;
        g_grid[dev][ilp] = grid;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    return CG_OK;
}

bool row_is_perm(const uint8_t* g, int n) {
    unsigned seen = 0;
    for (int i = 0; i < n; ++i) {
        if (g[i] >= n || (seen >> g[i]) & 1u) return false;
        seen |= 1u << g[i];
    }
    return true;
}

bool row_is_identity(const uint8_t* g, int n) {
    for (int i = 0; i < n; ++i)
        if (g[i] != i) return false;
    return true;
}

bool rows_equal(const uint8_t* a, const uint8_t* b, int n) {
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return false;
    return true;
}

// Shift-and-mask form of the gather t[i] = s[g[i]] on 4-bit elements (every permutation of
// n <= 16 elements has at most 16 distinct offsets i - g[i]).
void make_gensm(const uint8_t* g, int n, cg::GenSM& G) {
    std::memset(&G, 0, sizeof(G));
    G.width = 4;
    for (int i = 0; i < n; ++i) {
        const unsigned rot = (unsigned)((4 * (i - (int)g[i]) + 64) & 63);
        uint32_t t = 0;
        while (t < G.nterms && G.rot[t] != rot) ++t;
        if (t == G.nterms) {
            G.rot[t] = (uint8_t)rot;
            G.nterms++;
        }
        G.mask[t] |= 0xFull << (4 * i);
    }
}

// Host staging (the call holds g_mu while it uses them; fixed arrays, no heap): the distinct
// non-identity rows and their device form.
uint8_t g_rows[kMaxGens][cg::kMaxN];
cg::GenSM g_host_gens[kMaxGens];

// Distinct non-identity rows of gens into g_rows; returns their number, or -1 when there are
// more than kMaxGens of them.
int distinct_rows(const uint8_t* gens, int k, int n) {
    int kk = 0;
    for (int j = 0; j < k; ++j) {
        const uint8_t* r = gens + (size_t)j * n;
        if (row_is_identity(r, n)) continue;
        bool dup = false;
        for (int m = 0; m < kk && !dup; ++m) dup = rows_equal(g_rows[m], r, n);
        if (dup) continue;
        if (kk == kMaxGens) return -1;
        std::memcpy(g_rows[kk++], r, n);
    }
    return kk;
}

// Each generator's parent-edge tag: 1 + index of its inverse among the rows when that index is
// below 15 (the tag lives in key bits 60-63), else 0 (no skip).
void set_inverse_tags(int kk, int n) {
    for (int j = 0; j < kk; ++j) {
        uint8_t inv[cg::kMaxN];
        for (int i = 0; i < n; ++i) inv[g_rows[j][i]] = (uint8_t)i;
        g_host_gens[j].inv_tag = 0;
        for (int m = 0; m < kk && m < 15; ++m)
            if (rows_equal(g_rows[m], inv, n)) { g_host_gens[j].inv_tag = (uint32_t)(m + 1); break; }
    }
}

bool closed_under_inverse(int kk, int n) {
    for (int j = 0; j < kk; ++j) {
        uint8_t inv[cg::kMaxN];
        for (int i = 0; i < n; ++i) inv[g_rows[j][i]] = (uint8_t)i;
        bool found = false;
        for (int m = 0; m < kk && !found; ++m) found = rows_equal(g_rows[m], inv, n);
        if (!found) return false;
    }
    return true;
}

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return CG_OK;
    cudaGetLastError();
    return CG_ECUDA;
}

// Once work is enqueued on the stream, every return waits for it first: the shared array must
// be idle when the next call (possibly on another stream) takes the lock.
struct StreamDrain {
    cudaStream_t st;
    bool armed = false;
    ~StreamDrain() {
        if (armed && cudaStreamSynchronize(st) != cudaSuccess) cudaGetLastError();
    }
};

}  // namespace

extern "C" int cg_growth_run_noalloc(int n, int k, const uint8_t* gens, int inverse_closed,
                                     int max_radius, void* cuda_stream,
                                     uint64_t* layer_sizes_out, int cap, int* num_layers_out) {
    if (n < 1 || n > cg::kMaxN || k < 1 || !gens || !layer_sizes_out || !num_layers_out || cap < 1)
        return CG_EINVAL;
    for (int j = 0; j < k; ++j)
        if (!row_is_perm(gens + (size_t)j * n, n)) return CG_EINVAL;

    std::lock_guard<std::mutex> lock(g_mu);
    // identity rows add no edge and duplicates add none either; the limit counts distinct rows
    const int kk = distinct_rows(gens, k, n);
    if (kk < 0) return CG_ETOOBIG;
    if (inverse_closed && !closed_under_inverse(kk, n)) return CG_ENOTCLOSED;
    if (kk == 0 || max_radius == 0) {
        *num_layers_out = 1;
        layer_sizes_out[0] = 1;
        return kk == 0 ? CG_OK : CG_TRUNC_RADIUS;
    }
    for (int j = 0; j < kk; ++j) make_gensm(g_rows[j], n, g_host_gens[j]);
    set_inverse_tags(kk, n);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_rc(e);
    int rc = setup_device(dev);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* base = g_scratch_addr[dev];
    uint64_t* keys = reinterpret_cast<uint64_t*>(base + kOffKeys);
    uint64_t* table = reinterpret_cast<uint64_t*>(base + kOffTable);
    uint64_t* layers = reinterpret_cast<uint64_t*>(base + kOffLayers);
    cg::GenSM* d_gens = reinterpret_cast<cg::GenSM*>(base + kOffGens);
    cg::JobDev* d_job = reinterpret_cast<cg::JobDev*>(base + kOffJob);
    cg::Ctl* d_ctl = reinterpret_cast<cg::Ctl*>(base + kOffCtl);
    unsigned long long* d_ubeg = reinterpret_cast<unsigned long long*>(base + kOffUbeg);

    cg::JobDev J;
    std::memset(&J, 0, sizeof(J));
    J.keys = keys;
    J.keys_cap = kMaxStates;
    J.table = table;
    J.table_mask = kTableSlots - 1;
    J.gens = d_gens;
    J.layer_sizes = layers;
    J.k = kk;
    J.n = n;
    J.layers_cap = cg::kMaxLayers;
    J.max_radius = max_radius < 0 ? -1 : max_radius;
    J.tagged = n <= 15 ? 1 : 0;

    // Probe ILP and grid as the allocating path chooses them for a hash table: all generators
    // in flight up to 4, and fewer blocks for small groups (at most n! states, which is also
    // the bound for any subgroup), so that a small growth does not pay a barrier across every
    // co-resident block on each layer.
    const int ilp = kk < 4 ? kk : 4;
    uint64_t bound = 1;
    for (int i = 2; i <= n && bound < kMaxStates; ++i) bound *= (uint64_t)i;
    if (bound > kMaxStates) bound = kMaxStates;
    const uint64_t want = bound / 512 + 1;
    const int grid = (int)(want < (uint64_t)g_grid[dev][ilp] ? want : (uint64_t)g_grid[dev][ilp]);

    // Everything the kernels read first is rewritten here: the visited table is emptied, the
    // control block zeroed, the job and generators uploaded.
    StreamDrain drain{st};
    drain.armed = true;
    if ((e = cudaMemcpyAsync(d_gens, g_host_gens, sizeof(cg::GenSM) * kk, cudaMemcpyHostToDevice, st)))
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st))) return cuda_rc(e);
    if ((e = cudaMemsetAsync(table, 0xFF, kTableSlots * 8, st))) return cuda_rc(e);
    if ((e = cudaMemsetAsync(d_ctl, 0, sizeof(cg::Ctl), st))) return cuda_rc(e);
    if ((e = cg::launch_init_jobs(d_job, 1, d_ubeg, d_ctl, st))) return cuda_rc(e);
    if ((e = cg::launch_hash_grow(d_job, 1, d_ubeg, d_ctl, grid, cg::kMaxLayers + 1, kTimeoutNs,
                                  ilp, st, 0, nullptr, &J)))
        return cuda_rc(e);
    cg::Ctl ctl;
    if ((e = cudaMemcpyAsync(&J, d_job, sizeof(J), cudaMemcpyDeviceToHost, st))) return cuda_rc(e);
    if ((e = cudaMemcpyAsync(&ctl, d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st))) return cuda_rc(e);
    if ((e = cudaStreamSynchronize(st))) return cuda_rc(e);
    if (ctl.err) return ctl.err;
    if (J.status == cg::kNeedMem) return CG_ETOOBIG;   // more states than the scratch holds
    const int nl = J.radius + 1;
    *num_layers_out = nl;
    if (cap < nl) return CG_EINVAL;
    if ((e = cudaMemcpyAsync(layer_sizes_out, layers, sizeof(uint64_t) * nl, cudaMemcpyDeviceToHost, st)))
        return cuda_rc(e);
    if ((e = cudaStreamSynchronize(st))) return cuda_rc(e);
    drain.armed = false;
    switch (J.status) {
        case cg::kDone: return CG_OK;
        case cg::kTruncRadius: return CG_TRUNC_RADIUS;
        case cg::kTruncAbove: return CG_TRUNC_ABOVE;
        default: return CG_EDEVICE;
    }
}
