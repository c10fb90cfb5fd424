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
// once per device with cudaGetSymbolAddress and passed to the kernels.
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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on the
// first call for that device, with that device current).
int scratch_address(void** out)
{
    int dev = 0;
    LM_CUDA(cudaGetDevice(&dev));
    LM_CHECK(dev >= 0 && dev < kMaxDevices, LM_ERR_INVALID_ARG, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        LM_CHECK(e == cudaSuccess && p != nullptr, LM_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed: %s",
                 cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
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
