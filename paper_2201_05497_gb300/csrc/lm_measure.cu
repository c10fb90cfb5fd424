// Measurement utilities used only by the benchmark (declared in
// include/lm_measure.h, not part of the LM-SPDHG interface of lmspdhg.h):
// L2 and shared-memory throughput probes that give the benchmark's in-run
// peaks for gather/atomic traffic, and exact traversal statistics (samples
// and in-grid neighbour touches) that give its algorithmic byte counts.
#include <algorithm>
#include <cstring>

#include "lm_internal.h"
#include "../../include/lm_measure.h"

using namespace lmh;
using namespace lmk;

namespace {

// ---- L2 throughput probes (measurement utility) ----
__device__ __forceinline__ unsigned hash32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Shared-memory probe: random 4-byte reads (mode 4) or float atomic adds
// (mode 5) on a 32 KB array per block, indices from a linear congruential
// sequence per thread (two instructions per index).
constexpr int SPROBE_N = 8192;
__global__ void __launch_bounds__(256) smem_probe_kernel(int mode, int iters, float* sink)
{
    __shared__ float sm[SPROBE_N];
    for (int k = threadIdx.x; k < SPROBE_N; k += blockDim.x) sm[k] = 0.0f;
    __syncthreads();
    unsigned idx = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u;
    float acc = 0.0f;
    if (mode == 4) {
        for (int it = 0; it < iters; ++it) {
#pragma unroll 8
            for (int r = 0; r < 64; ++r) {
                idx = idx * 1664525u + 1013904223u;
                acc += sm[idx >> 19];
            }
        }
    } else {
        for (int it = 0; it < iters; ++it) {
#pragma unroll 8
            for (int r = 0; r < 64; ++r) {
                idx = idx * 1664525u + 1013904223u;
                atomicAdd(sm + (idx >> 19), 1.0f);
            }
        }
        __syncthreads();
        acc = sm[threadIdx.x];
    }
    if (acc == 12345.678f) *sink = acc;
}

__global__ void __launch_bounds__(256) probe_kernel(float* buf, size_t n, int mode, int iters, float* sink)
{
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    float acc = 0.0f;
    const size_t mask = n - 1;  // n is a power of two
    for (int it = 0; it < iters; ++it) {
        if (mode == 0) {
            const float4* b4 = reinterpret_cast<const float4*>(buf);
            for (size_t i = tid; i < n / 4; i += nth) {
                const float4 v = __ldcg(b4 + i);
                acc += v.x + v.y + v.z + v.w;
            }
        } else if (mode == 1) {
            for (size_t i = tid; i < n; i += nth) atomicAdd(buf + i, 1.0f);
        } else if (mode == 2) {
            for (size_t i = tid; i < n; i += nth) acc += __ldcg(buf + (hash32((unsigned)(i + it * 7919u)) & mask));
        } else {
            for (size_t i = tid; i < n; i += nth) atomicAdd(buf + (hash32((unsigned)(i + it * 7919u)) & mask), 1.0f);
        }
    }
    if (acc == 12345.678f) *sink = acc;
}

}  // namespace

extern "C" {

int lm_probe_l2(void* buf, size_t bytes, int32_t mode, int32_t iters, double* gbs_out, void* stream)
{
    clear_error();
    LM_CHECK(buf && gbs_out && bytes >= 4096 && mode >= 0 && mode <= 5 && iters >= 1, LM_ERR_INVALID_ARG,
             "bad probe arguments");
    if (mode >= 4) {
        cudaStream_t st = S(stream);
        int bps = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, smem_probe_kernel, 256, 0);
        const int grid = std::max(1, bps) * num_sms();
        smem_probe_kernel<<<grid, 256, 0, st>>>(mode, 1, (float*)buf);  // warm-up
        cudaEvent_t e0, e1;
        LM_CUDA(cudaEventCreate(&e0));
        LM_CUDA(cudaEventCreate(&e1));
        cudaEventRecord(e0, st);
        smem_probe_kernel<<<grid, 256, 0, st>>>(mode, iters, (float*)buf);
        cudaEventRecord(e1, st);
        count_launch(2);
        cudaError_t ce = cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "probe failed: %s", cudaGetErrorString(ce));
        *gbs_out = (double)grid * 256.0 * 64.0 * iters * 4.0 / (ms * 1e-3) / 1e9;
        return LM_OK;
    }
    size_t n = 1024;
    while (n * 2 * 4 <= bytes) n *= 2;  // power-of-two float count
    cudaStream_t st = S(stream);
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, probe_kernel, 256, 0);
    const int grid = std::max(1, bps) * num_sms();
    float* f = (float*)buf;
    LM_CUDA(cudaMemsetAsync(buf, 0, n * 4, st));
    probe_kernel<<<grid, 256, 0, st>>>(f, n, mode, 1, f);  // warm L2
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    probe_kernel<<<grid, 256, 0, st>>>(f, n, mode, iters, f);
    cudaEventRecord(e1, st);
    count_launch(2);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "probe failed: %s", cudaGetErrorString(ce));
    *gbs_out = (double)n * 4.0 * iters / (ms * 1e-3) / 1e9;
    return LM_OK;
}

int lm_traversal_stats(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
                       void* ws, size_t ws_bytes, int64_t* n_samples, int64_t* n_touches, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    LM_CHECK(ev != nullptr && ev->n >= 0, LM_ERR_INVALID_ARG, "events are NULL or negative");
    LM_CHECK(ev->n == 0 || (ev->det1 && ev->det2), LM_ERR_INVALID_ARG, "event detector arrays are NULL");
    LM_CHECK(n_samples && n_touches, LM_ERR_INVALID_ARG, "NULL output");
    LM_CHECK(ws != nullptr && ws_bytes >= 16, LM_ERR_NOMEM, "statistics need 16 workspace bytes");
    *n_samples = 0;
    *n_touches = 0;
    if (ev->n == 0) return LM_OK;
    cudaStream_t st = S(stream);
    unsigned long long* cnt = (unsigned long long*)ws;
    LM_CUDA(cudaMemsetAsync(cnt, 0, 16, st));
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = G;
    a.det1 = ev->det1;
    a.det2 = ev->det2;
    a.tof = ev->tof;
    a.e_begin = 0;
    a.e_end = ev->n;
    a.chunk = 32;
    a.acci_std = cnt;
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;
    rc = launch_events(EV_COUNT, two_d, a, ev_grid(EV_COUNT, two_d), st);
    unsigned long long h[2] = {0, 0};
    cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, st);
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(rc == LM_OK, rc, "statistics launch failed");
    *n_samples = (int64_t)h[0];
    *n_touches = (int64_t)h[1];
    return LM_OK;
}

}  // extern "C"
