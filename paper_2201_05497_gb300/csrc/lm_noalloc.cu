// Deterministic back-projection for callers that cannot allocate device
// memory or hand the library a workspace.
//
// Some callers cannot allocate: a plug-in whose host application owns all
// device memory and allows no further allocations, or a real-time path that
// must not allocate after start-up (cudaMalloc may synchronise the device
// and its latency is unbounded).  For them this file keeps the scratch of
// the fixed-point back-projection in a file-scope device array of fixed
// size, instead of in a caller workspace.
//
// The array is allocated by the CUDA runtime when the module is loaded on a
// GPU and stays allocated on every GPU that loads the library until the
// process exits.  Host code must not use the array's name as an address
// (in host code it is only a stand-in); the device address is looked up
// once per CUDA context with cudaGetSymbolAddress and passed to the kernels.
#include <cstring>
#include <mutex>

#include "lm_internal.h"

namespace {

// Voxel capacity of the shared scratch: 2^22 = 4,194,304 voxels, enough for
// a 200 x 200 x 96 grid.  8 bytes per voxel (64-bit fixed-point sums, one
// image layout) plus 32 words for the max-|value| bits: 32 MiB + 256 B.
constexpr int64_t kMaxVox = int64_t(1) << 22;
constexpr int64_t kTail = 32;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxVox + kTail];

using CtxGetCurrent = CUresult (*)(CUcontext*);
using CtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current CUDA context (0 when the thread
// has none yet).  The scratch is a module global, so its address belongs to
// the context that loaded the module: a context destroyed and created again
// (cudaDeviceReset, or a re-created primary context) loads the module anew,
// possibly at another address.  Context ids are unique within the process
// and never reused, unlike context handles.
int current_context_id(unsigned long long* id)
{
    static CtxGetCurrent get_cur = nullptr;
    static CtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(p);
    });
    LM_CHECK(get_cur != nullptr && get_id != nullptr, LM_ERR_CUDA,
             "cuCtxGetCurrent / cuCtxGetId are not available from the driver");
    *id = 0;
    CUcontext ctx = nullptr;
    CUresult r = get_cur(&ctx);
    LM_CHECK(r == CUDA_SUCCESS, LM_ERR_CUDA, "cuCtxGetCurrent failed (%d)", (int)r);
    if (ctx == nullptr) return LM_OK;
    r = get_id(ctx, id);
    LM_CHECK(r == CUDA_SUCCESS && *id != 0, LM_ERR_CUDA, "cuCtxGetId failed (%d)", (int)r);
    return LM_OK;
}

constexpr int kMaxContexts = 64;
std::mutex g_mu;
unsigned long long g_ctx[kMaxContexts] = {};
void* g_addr[kMaxContexts] = {};
int g_n = 0;  // entries in use; when full, the oldest entry is replaced
int g_next = 0;

// Device address of the scratch in the current context, looked up with
// cudaGetSymbolAddress on the first call made in that context (with its
// device current) and cached under the context's id.
int scratch_address(void** out)
{
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; id != 0 && i < g_n; ++i)
        if (g_ctx[i] == id) {
            *out = g_addr[i];
            return LM_OK;
        }
    // first call in this context: cudaGetSymbolAddress also makes the runtime
    // bind the device's primary context when the thread had none
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    LM_CHECK(e == cudaSuccess && p != nullptr, LM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed: %s",
             cudaGetErrorString(e));
    if (id == 0) {
        rc = current_context_id(&id);
        if (rc) return rc;
        LM_CHECK(id != 0, LM_ERR_CUDA, "no current CUDA context after the symbol lookup");
    }
    const int slot = g_n < kMaxContexts ? g_n++ : g_next;
    if (g_n == kMaxContexts) g_next = (slot + 1) % kMaxContexts;
    g_ctx[slot] = id;
    g_addr[slot] = p;
    *out = p;
    return LM_OK;
}

}  // namespace

using namespace lmh;

extern "C" {

int lm_back_deterministic_noalloc(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                                  const lm_events* ev, const float* v, float* img, void* stream)
{
    clear_error();
    lmk::Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    LM_CHECK(ev != nullptr && ev->n >= 0, LM_ERR_INVALID_ARG, "events are NULL or negative");
    LM_CHECK(nvox(grid) <= kMaxVox, LM_ERR_NOMEM,
             "grid has %lld voxels; the workspace-free back-projection supports at most %lld",
             (long long)nvox(grid), (long long)kMaxVox);
    if (ev->n == 0) return LM_OK;
    LM_CHECK(ev->det1 && ev->det2, LM_ERR_INVALID_ARG, "event detector arrays are NULL");
    LM_CHECK(v != nullptr && img != nullptr, LM_ERR_INVALID_ARG, "v or img is NULL");
    LM_CHECK(tof->n_bins == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = S(stream);
    unsigned long long* acc = (unsigned long long*)base;
    unsigned* maxbits = (unsigned*)(acc + kMaxVox);
    // the array keeps the previous call's contents: clear what must start at zero
    LM_CUDA(cudaMemsetAsync(acc, 0, (size_t)nvox(grid) * 8, st));
    LM_CUDA(cudaMemsetAsync(maxbits, 0, kTail * 8, st));
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = G;
    a.det1 = ev->det1;
    a.det2 = ev->det2;
    a.tof = ev->tof;
    a.corr = ev->corr;
    a.vin = v;
    a.e_begin = 0;
    a.e_end = ev->n;
    a.chunk = 32;
    a.stepmax = 2.0f * std::fmax(grid->h[0], std::fmax(grid->h[1], grid->h[2]));
    a.maxbits = maxbits;
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;
    rc = launch_events(EV_ABSMAX, two_d, a, ev_grid(EV_ABSMAX, two_d), st);
    LM_CHECK(rc == LM_OK, rc, "max reduction launch failed");
    a.acci_std = acc;  // one layout: y-principal LORs scatter with the x-fastest strides
    rc = launch_events(EV_BACK_FX, two_d, a, ev_grid(EV_BACK_FX, two_d), st);
    LM_CHECK(rc == LM_OK, rc, "fixed-point back-projection launch failed");
    launch_fold_fixed(grid, img, acc, nullptr, maxbits, (long long)ev->n, a.stepmax, st);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

}  // extern "C"
