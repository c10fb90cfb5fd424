// Event set-up of Alg. 2: validation, the event counts mu_e and the split
// of the list into n sub lists, event e to subset e mod n.
//
// mu_e counts the events of the whole list in e's data bin (unordered
// detector pair + TOF bin signed toward the larger detector id).  The count
// uses an open-addressing hash table on the packed 64-bit bin key
// (insert-or-increment with atomicCAS / atomicAdd), which gives exact
// integer counts independent of thread order.  The subset-contiguous copy is
// a gather: output position p is decoded into (subset k, rank r) and reads
// event r*n + k.
#include <cstring>
#include <vector>

#include "lm_internal.h"

namespace {

constexpr unsigned long long EMPTY = ~0ULL;

__device__ __forceinline__ unsigned long long mix64(unsigned long long k)
{
    // 64-bit finaliser of MurmurHash3 (Appleby)
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ unsigned long long bin_key(int d1, int d2, int t)
{
    const bool sw = d1 > d2;
    const unsigned long long lo = (unsigned)(sw ? d2 : d1), hi = (unsigned)(sw ? d1 : d2);
    const int tc = sw ? -t : t;
    return (lo << 36) | (hi << 8) | (unsigned long long)(tc + 127);
}

enum { ERR_RANGE = 1, ERR_DOMAIN = 2, ERR_MU = 4, ERR_TABLE = 8 };

__global__ void validate_insert(const int32_t* __restrict__ d1, const int32_t* __restrict__ d2,
                                const int16_t* __restrict__ tb, const float* __restrict__ corr,
                                const float* __restrict__ contam, int64_t n, int n_det, int tof_on, int M,
                                unsigned long long* keys, unsigned* counts, unsigned long long mask, unsigned* err,
                                unsigned long long* bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = d1[e], b = d2[e];
        const int t = (tof_on && tb) ? (int)tb[e] : 0;
        unsigned f = 0;
        if (a < 0 || a >= n_det || b < 0 || b >= n_det || a == b) f |= ERR_RANGE;
        if (tof_on && (t < -M || t > M)) f |= ERR_RANGE;
        if (corr && !(corr[e] > 0.0f)) f |= ERR_DOMAIN;
        if (contam && !(contam[e] > 0.0f)) f |= ERR_DOMAIN;
        if (f) {
            atomicOr(err, f);
            atomicMin(bad, (unsigned long long)e);
            continue;
        }
        const unsigned long long key = bin_key(a, b, t);
        unsigned long long slot = mix64(key) & mask;
        bool done = false;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(keys + slot, EMPTY, key);
            if (prev == EMPTY || prev == key) {
                atomicAdd(counts + slot, 1u);
                done = true;
                break;
            }
            slot = (slot + 1) & mask;
        }
        if (!done) atomicOr(err, (unsigned)ERR_TABLE);
    }
}

__device__ __forceinline__ unsigned lookup(const unsigned long long* keys, const unsigned* counts,
                                           unsigned long long mask, unsigned long long key)
{
    unsigned long long slot = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[slot];
        if (k == key) return counts[slot];
        if (k == EMPTY) return 0u;
        slot = (slot + 1) & mask;
    }
    return 0u;
}

__global__ void permute_events(const int32_t* __restrict__ d1, const int32_t* __restrict__ d2,
                               const int16_t* __restrict__ tb, const float* __restrict__ corr,
                               const float* __restrict__ contam, int64_t n, int n_sub, int tof_on,
                               const unsigned long long* keys, const unsigned* counts, unsigned long long mask,
                               int32_t* o1, int32_t* o2, int16_t* ot, float* oc, float* os, uint16_t* omu,
                               unsigned* err)
{
    const int64_t q = n / n_sub, r = n % n_sub;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        int64_t k, rank;
        if (p < r * (q + 1)) {
            k = p / (q + 1);
            rank = p - k * (q + 1);
        } else {
            const int64_t p2 = p - r * (q + 1);
            k = r + p2 / q;
            rank = p2 - (k - r) * q;
        }
        const int64_t e = rank * n_sub + k;
        const int a = d1[e], b = d2[e];
        const int t = (tof_on && tb) ? (int)tb[e] : 0;
        o1[p] = a;
        o2[p] = b;
        if (ot) ot[p] = (int16_t)t;
        if (oc) oc[p] = corr ? corr[e] : 1.0f;
        if (os) os[p] = contam ? contam[e] : 0.0f;
        const unsigned c = lookup(keys, counts, mask, bin_key(a, b, t));
        if (c > 65535u || c == 0u) atomicOr(err, (unsigned)(c == 0u ? ERR_TABLE : ERR_MU));
        omu[p] = (uint16_t)(c > 65535u ? 65535u : c);
    }
}

size_t table_cap(int64_t n)
{
    size_t cap = 1024;
    while (cap < (size_t)(2 * n)) cap <<= 1;
    return cap;
}

}  // namespace

using namespace lmh;

extern "C" {

size_t lm_setup_workspace_bytes(int64_t n_events)
{
    if (n_events < 0) return 0;
    const size_t cap = table_cap(n_events);
    return align_up(cap * 8) + align_up(cap * 4) + 256;
}

int lm_event_setup(const lm_scanner* sc, const lm_tof* tof, const lm_events* ev, int32_t n_subsets,
                   int32_t* det1_out, int32_t* det2_out, int16_t* tof_out, float* corr_out, float* contam_out,
                   uint16_t* mu_out, int64_t* sub_off_host, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    LM_CHECK(sc != nullptr && tof != nullptr && ev != nullptr, LM_ERR_INVALID_ARG, "NULL descriptor");
    LM_CHECK(sc->n_rings >= 1 && sc->n_xtal >= 2, LM_ERR_INVALID_ARG, "bad scanner");
    LM_CHECK((int64_t)sc->n_rings * sc->n_xtal < (int64_t(1) << 27), LM_ERR_INVALID_ARG, "too many crystals");
    LM_CHECK(n_subsets >= 1, LM_ERR_INVALID_ARG, "n_subsets must be >= 1");
    LM_CHECK(ev->n >= 0, LM_ERR_INVALID_ARG, "negative event count");
    LM_CHECK(sub_off_host != nullptr, LM_ERR_INVALID_ARG, "sub_off_host is NULL");
    LM_CHECK(tof->n_bins == 0 || (tof->n_bins % 2 == 1 && tof->n_bins <= 255), LM_ERR_INVALID_ARG,
             "n_bins must be 0 or odd <= 255");
    const int64_t n = ev->n;
    const int64_t q = n / n_subsets, r = n % n_subsets;
    for (int64_t k = 0; k <= n_subsets; ++k) sub_off_host[k] = k * q + (k < r ? k : r);
    if (n == 0) return LM_OK;
    LM_CHECK(ev->det1 && ev->det2 && det1_out && det2_out && mu_out, LM_ERR_INVALID_ARG, "NULL event array");
    LM_CHECK(tof->n_bins == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    const size_t need = lm_setup_workspace_bytes(n);
    LM_CHECK(ws != nullptr && ws_bytes >= need, LM_ERR_NOMEM, "event set-up needs %zu workspace bytes", need);
    cudaStream_t st = S(stream);
    const size_t cap = table_cap(n);
    char* w = (char*)ws;
    unsigned long long* keys = (unsigned long long*)w;
    unsigned* counts = (unsigned*)(w + align_up(cap * 8));
    unsigned* err = (unsigned*)(w + align_up(cap * 8) + align_up(cap * 4));
    unsigned long long* bad = (unsigned long long*)(err + 2);
    LM_CUDA(cudaMemsetAsync(keys, 0xff, cap * 8, st));
    LM_CUDA(cudaMemsetAsync(counts, 0, cap * 4, st));
    LM_CUDA(cudaMemsetAsync(err, 0, 8, st));
    LM_CUDA(cudaMemsetAsync(bad, 0xff, 8, st));
    const int n_det = sc->n_rings * sc->n_xtal;
    const int tof_on = tof->n_bins > 0;
    const int M = tof_on ? (tof->n_bins - 1) / 2 : 0;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16));
    validate_insert<<<grid, 256, 0, st>>>(ev->det1, ev->det2, ev->tof, ev->corr, ev->contam, n, n_det, tof_on, M, keys,
                                          counts, (unsigned long long)(cap - 1), err, bad);
    count_launch();
    LM_CUDA(cudaGetLastError());
    unsigned herr = 0;
    unsigned long long hbad = 0;
    LM_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(&hbad, bad, 8, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(!(herr & ERR_RANGE), LM_ERR_OUT_OF_RANGE, "event %llu: detector id or TOF bin out of range",
             (unsigned long long)hbad);
    LM_CHECK(!(herr & ERR_DOMAIN), LM_ERR_DOMAIN, "event %llu: corr and contam must be > 0",
             (unsigned long long)hbad);
    LM_CHECK(!(herr & ERR_TABLE), LM_ERR_CUDA, "event count table overflow");
    permute_events<<<grid, 256, 0, st>>>(ev->det1, ev->det2, ev->tof, ev->corr, ev->contam, n, n_subsets, tof_on,
                                         keys, counts, (unsigned long long)(cap - 1), det1_out, det2_out, tof_out,
                                         corr_out, contam_out, mu_out, err);
    count_launch();
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(!(herr & ERR_MU), LM_ERR_OUT_OF_RANGE, "an event count exceeds 65535");
    LM_CHECK(!(herr & ERR_TABLE), LM_ERR_CUDA, "event count lookup failed");
    return LM_OK;
}

}  // extern "C"
