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
int g_grid[64] = {};

// Once per device, with that device current: the device address of the scratch array (the
// array's name in host code is only a host-side stand-in, not a device address).
int setup_device(int dev) {
    if (dev < 0 || dev >= 64) return CG_EINVAL;
    if (g_scratch_addr[dev]) return CG_OK;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return CG_ECUDA;
    }
    const int grid = cg::hash_grow_max_grid(dev, 1, false);
    if (grid <= 0) return CG_ECUDA;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    g_grid[dev] = grid;
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

bool has_inverse(const uint8_t* gens, int k, int n, int j) {
    for (int m = 0; m < k; ++m) {
        bool inv = true;
        for (int i = 0; i < n && inv; ++i) inv = gens[m * n + gens[j * n + i]] == i;
        if (inv) return true;
    }
    return false;
}

void make_gensm(const uint8_t* g, int n, cg::GenSM& G) {
    std::memset(&G, 0, sizeof(G));
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

// Host staging for the uploads (the call holds g_mu while it uses them).
cg::GenSM g_host_gens[kMaxGens];

int cuda_rc(cudaError_t e) {
    if (e == cudaSuccess) return CG_OK;
    cudaGetLastError();
    return CG_ECUDA;
}

}  // namespace

extern "C" int cg_growth_run_noalloc(int n, int k, const uint8_t* gens, int inverse_closed,
                                     int max_radius, void* cuda_stream,
                                     uint64_t* layer_sizes_out, int cap, int* num_layers_out) {
    if (n < 1 || n > cg::kMaxN || k < 1 || !gens || !layer_sizes_out || !num_layers_out || cap < 1)
        return CG_EINVAL;
    if (k > kMaxGens) return CG_ETOOBIG;
    for (int j = 0; j < k; ++j)
        if (!row_is_perm(gens + j * n, n)) return CG_EINVAL;
    if (inverse_closed)
        for (int j = 0; j < k; ++j)
            if (!has_inverse(gens, k, n, j)) return CG_ENOTCLOSED;

    std::lock_guard<std::mutex> lock(g_mu);
    int kk = 0;
    for (int j = 0; j < k; ++j)
        if (!row_is_identity(gens + j * n, n)) make_gensm(gens + j * n, n, g_host_gens[kk++]);
    if (kk == 0 || max_radius == 0) {
        *num_layers_out = 1;
        layer_sizes_out[0] = 1;
        return kk == 0 ? CG_OK : CG_TRUNC_RADIUS;
    }

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

    // Everything the kernels read first is rewritten here: the visited table is emptied, the
    // control block zeroed, the job and generators uploaded.
    if ((e = cudaMemcpyAsync(d_gens, g_host_gens, sizeof(cg::GenSM) * kk, cudaMemcpyHostToDevice, st)))
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(d_job, &J, sizeof(J), cudaMemcpyHostToDevice, st))) return cuda_rc(e);
    if ((e = cudaMemsetAsync(table, 0xFF, kTableSlots * 8, st))) return cuda_rc(e);
    if ((e = cudaMemsetAsync(d_ctl, 0, sizeof(cg::Ctl), st))) return cuda_rc(e);
    if ((e = cg::launch_init_jobs(d_job, 1, d_ubeg, d_ctl, st))) return cuda_rc(e);
    if ((e = cg::launch_hash_grow(d_job, 1, d_ubeg, d_ctl, g_grid[dev], cg::kMaxLayers + 1,
                                  kTimeoutNs, 1, st)))
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
    switch (J.status) {
        case cg::kDone: return CG_OK;
        case cg::kTruncRadius: return CG_TRUNC_RADIUS;
        case cg::kTruncAbove: return CG_TRUNC_ABOVE;
        default: return CG_EDEVICE;
    }
}
