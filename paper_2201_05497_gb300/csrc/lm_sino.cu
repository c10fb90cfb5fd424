// Sinogram SPDHG (Alg. 1): the bins of a TOF sinogram laid out as the
// event list of the LM-SPDHG state (lm_params.sinogram = 1).  Every bin
// (canonical LOR l, TOF bin m) becomes one "event" with its count d_b in
// place of the listmode multiplicity, its contamination s_b and the LOR's
// multiplicative factor; Alg. 1's dual step then differs from Alg. 2's only
// in the prox parameter (S_b d_b) and in back-projecting y+ - y undivided.
// Empty bins are processed like every other bin (they keep y = 1).
//
// Subsets are views: LORs with the same (c1 + c2) mod n_xtal are parallel,
// and view v goes to subset v mod n.  Bins are written subset by subset, in
// canonical order inside a subset.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lm_internal.h"

using namespace lmh;

namespace {

void pair_of_q(int64_t q, int n_xtal, int& c1, int& c2)
{
    const int64_t B = (int64_t)n_xtal * ((n_xtal - 1) / 2);
    if (q < B) {
        c1 = (int)(q % n_xtal);
        c2 = (int)((c1 + 1 + q / n_xtal) % n_xtal);
    } else {
        c1 = (int)(q - B);
        c2 = c1 + n_xtal / 2;
    }
}

__global__ void __launch_bounds__(256) sino_bins_kernel(int n_xtal, int n_rings, int nb, int M, int64_t n_pairs,
                                                        const int* __restrict__ qsub, const int* __restrict__ qrank,
                                                        const int64_t* __restrict__ off, const uint16_t* __restrict__ d,
                                                        const float* __restrict__ s, const float* __restrict__ lf,
                                                        int32_t* det1, int32_t* det2, int16_t* tof, float* corr,
                                                        float* contam, uint16_t* mu, unsigned* bad)
{
    const int64_t nr2 = (int64_t)n_rings * n_rings;
    const int64_t total = n_pairs * nr2 * nb;
    const int64_t B = (int64_t)n_xtal * ((n_xtal - 1) / 2);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < total; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = b / nb;
        const int mi = (int)(b - l * nb);
        const int64_t q = l / nr2;
        const int rr = (int)(l - q * nr2);
        const int r1 = rr / n_rings, r2 = rr - r1 * n_rings;
        int c1, c2;
        if (q < B) {
            c1 = (int)(q % n_xtal);
            c2 = (int)((c1 + 1 + q / n_xtal) % n_xtal);
        } else {
            c1 = (int)(q - B);
            c2 = c1 + n_xtal / 2;
        }
        const int k = qsub[q];
        const int64_t pos = off[k] + ((int64_t)qrank[q] * nr2 + rr) * nb + mi;
        const float sb = s[b];
        if (!(sb > 0.0f) || !isfinite(sb)) atomicOr(bad, 1u);
        det1[pos] = r1 * n_xtal + c1;
        det2[pos] = r2 * n_xtal + c2;
        if (tof) tof[pos] = (int16_t)(mi - M);
        corr[pos] = lf ? lf[l] : 1.0f;
        contam[pos] = sb;
        mu[pos] = d[b];
    }
}

// +1 on a 16-bit count (the containing aligned 32-bit word by compare-and-
// swap); false at 65535 or after a bounded number of lost races.
__device__ __forceinline__ bool inc_u16(uint16_t* p)
{
    unsigned* w = reinterpret_cast<unsigned*>(reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)3);
    const unsigned sh = (reinterpret_cast<uintptr_t>(p) & 2) ? 16u : 0u;
    unsigned old = *w;
    for (int it = 0; it < (1 << 20); ++it) {
        if (((old >> sh) & 0xffffu) == 0xffffu) return false;
        const unsigned prev = atomicCAS(w, old, old + (1u << sh));
        if (prev == old) return true;
        old = prev;
    }
    return false;
}

// Counts of the events in every bin, in the subset order of lm_sino_setup.
// bad bit 1: an invalid event; bit 2: a count above 65535.
__global__ void __launch_bounds__(256) sino_count_kernel(int n_xtal, int n_rings, int nb, int M, const int32_t* det1,
                                                         const int32_t* det2, const int16_t* tbin, int64_t n,
                                                         const int* __restrict__ qsub, const int* __restrict__ qrank,
                                                         const int64_t* __restrict__ off, uint16_t* d, unsigned* bad)
{
    const int n_det = n_xtal * n_rings;
    const int64_t nr2 = (int64_t)n_rings * n_rings;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int a = det1[e], b = det2[e];
        const int m = tbin ? (int)tbin[e] : 0;
        if (a < 0 || b < 0 || a >= n_det || b >= n_det || m < -M || m > M) {
            atomicOr(bad, 1u);
            continue;
        }
        const int r1 = a / n_xtal, c1 = a - r1 * n_xtal, r2 = b / n_xtal, c2 = b - r2 * n_xtal;
        if (c1 == c2) {
            atomicOr(bad, 1u);
            continue;
        }
        // canonical pair and orientation (lm_sens's enumeration)
        const int off_c = ((c2 - c1) % n_xtal + n_xtal) % n_xtal;
        const int half = (n_xtal - 1) / 2;
        const bool direct = off_c >= 1 && off_c <= half;
        const bool even_mid = (n_xtal % 2 == 0) && off_c == n_xtal / 2;
        int64_t q;
        bool sw;
        if (even_mid) {
            q = (int64_t)n_xtal * half + min(c1, c2);
            sw = c1 > c2;
        } else if (direct) {
            q = (int64_t)(off_c - 1) * n_xtal + c1;
            sw = false;
        } else {
            q = (int64_t)(n_xtal - off_c - 1) * n_xtal + c2;
            sw = true;
        }
        const int ra = sw ? r2 : r1, rb = sw ? r1 : r2;
        const int mc = sw ? -m : m;
        const int64_t pos = off[qsub[q]] + ((int64_t)qrank[q] * nr2 + (int64_t)ra * n_rings + rb) * nb + (mc + M);
        if (!inc_u16(d + pos)) atomicOr(bad, 2u);
    }
}

struct SinoWs {
    int* qsub;
    int* qrank;
    int64_t* off;
    unsigned* bad;
};

size_t sino_ws_layout(const lm_scanner* sc, int n_subsets, SinoWs* w, void* base)
{
    const int64_t np = (int64_t)sc->n_xtal * (sc->n_xtal - 1) / 2;
    char* p = (char*)base;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* r = p ? p + o : nullptr;
        o += align_up(bytes);
        return r;
    };
    SinoWs t;
    t.qsub = (int*)take((size_t)np * 4);
    t.qrank = (int*)take((size_t)np * 4);
    t.off = (int64_t*)take((size_t)(n_subsets + 1) * 8);
    t.bad = (unsigned*)take(4);
    if (w) *w = t;
    return o;
}

// Host tables of the view-based subsets: subset and rank of every transaxial
// pair, the pairs of each subset in order, and the bin offsets.
void view_tables(int n_xtal, int n_subsets, int64_t per_q, std::vector<int>& qsub, std::vector<int>& qrank,
                 std::vector<int32_t>& qlist, std::vector<int64_t>& qoff, int64_t* sub_off)
{
    const int64_t np = (int64_t)n_xtal * (n_xtal - 1) / 2;
    qsub.assign((size_t)np, 0);
    qrank.assign((size_t)np, 0);
    std::vector<int64_t> cnt((size_t)n_subsets, 0);
    for (int64_t q = 0; q < np; ++q) {
        int c1, c2;
        pair_of_q(q, n_xtal, c1, c2);
        const int k = ((c1 + c2) % n_xtal) % n_subsets;
        qsub[(size_t)q] = k;
        qrank[(size_t)q] = (int)cnt[(size_t)k]++;
    }
    qoff.assign((size_t)n_subsets + 1, 0);
    for (int k = 0; k < n_subsets; ++k) qoff[(size_t)k + 1] = qoff[(size_t)k] + cnt[(size_t)k];
    qlist.assign((size_t)np, 0);
    for (int64_t q = 0; q < np; ++q) qlist[(size_t)(qoff[(size_t)qsub[(size_t)q]] + qrank[(size_t)q])] = (int32_t)q;
    sub_off[0] = 0;
    for (int k = 0; k < n_subsets; ++k) sub_off[k + 1] = sub_off[k] + cnt[(size_t)k] * per_q;
}

}  // namespace

extern "C" {

int64_t lm_sino_n_bins(const lm_scanner* sc, const lm_tof* tof)
{
    if (!sc || !tof) return 0;
    return lm_n_lor(sc) * std::max(1, (int)tof->n_bins);
}

size_t lm_sino_workspace_bytes(const lm_scanner* sc, int32_t n_subsets)
{
    if (!sc || sc->n_xtal < 2 || n_subsets < 1) return 0;
    return sino_ws_layout(sc, n_subsets, nullptr, nullptr);
}

int lm_sino_setup(const lm_scanner* sc, const lm_tof* tof, int32_t n_subsets, const uint16_t* d, const float* s,
                  const float* lor_factor, int32_t* det1_out, int32_t* det2_out, int16_t* tof_out, float* corr_out,
                  float* contam_out, uint16_t* d_out, int64_t* sub_off_host, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    LM_CHECK(sc && tof && sc->n_xtal >= 2 && sc->n_rings >= 1, LM_ERR_INVALID_ARG, "bad scanner");
    LM_CHECK(tof->n_bins >= 0 && (tof->n_bins == 0 || (tof->n_bins & 1)), LM_ERR_INVALID_ARG, "n_bins must be odd");
    LM_CHECK(n_subsets >= 1 && n_subsets < 65535, LM_ERR_INVALID_ARG, "n_subsets out of range");
    LM_CHECK(d && s && det1_out && det2_out && corr_out && contam_out && d_out && sub_off_host, LM_ERR_INVALID_ARG,
             "NULL argument");
    LM_CHECK(tof->n_bins == 0 || tof_out, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    const size_t need = sino_ws_layout(sc, n_subsets, nullptr, nullptr);
    LM_CHECK(ws != nullptr && ws_bytes >= need, LM_ERR_NOMEM, "sinogram set-up needs %zu workspace bytes", need);
    SinoWs W;
    sino_ws_layout(sc, n_subsets, &W, ws);
    const int n_xtal = sc->n_xtal;
    const int64_t np = (int64_t)n_xtal * (n_xtal - 1) / 2;
    const int nb = std::max(1, (int)tof->n_bins);
    const int64_t per_q = (int64_t)sc->n_rings * sc->n_rings * nb;
    // view of each transaxial pair, its subset and its rank inside the subset
    std::vector<int> qsub, qrank;
    std::vector<int32_t> qlist;
    std::vector<int64_t> qoff;
    view_tables(n_xtal, n_subsets, per_q, qsub, qrank, qlist, qoff, sub_off_host);
    cudaStream_t st = S(stream);
    LM_CUDA(cudaMemcpyAsync(W.qsub, qsub.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(W.qrank, qrank.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(W.off, sub_off_host, (size_t)(n_subsets + 1) * 8, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemsetAsync(W.bad, 0, 4, st));
    const int64_t total = np * per_q;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
    sino_bins_kernel<<<std::max(grid, 1), 256, 0, st>>>(n_xtal, sc->n_rings, nb, (nb - 1) / 2, np, W.qsub, W.qrank,
                                                        W.off, d, s, lor_factor, det1_out, det2_out,
                                                        tof->n_bins > 0 ? tof_out : nullptr, corr_out, contam_out,
                                                        d_out, W.bad);
    count_launch();
    LM_CUDA(cudaGetLastError());
    unsigned bad = 0;
    LM_CUDA(cudaMemcpyAsync(&bad, W.bad, 4, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(bad == 0, LM_ERR_DOMAIN, "every bin needs a finite contamination s_b > 0");
    return LM_OK;
}

int lm_sino_count(const lm_scanner* sc, const lm_tof* tof, int32_t n_subsets, const lm_events* ev, uint16_t* d_out,
                  int32_t* q_out, int64_t* qoff_out, int64_t* sub_off_host, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    LM_CHECK(sc && tof && ev && sc->n_xtal >= 2 && sc->n_rings >= 1, LM_ERR_INVALID_ARG, "bad scanner or events");
    LM_CHECK(tof->n_bins >= 0 && (tof->n_bins == 0 || (tof->n_bins & 1)), LM_ERR_INVALID_ARG, "n_bins must be odd");
    LM_CHECK(n_subsets >= 1 && n_subsets < 65535, LM_ERR_INVALID_ARG, "n_subsets out of range");
    LM_CHECK(d_out && q_out && qoff_out && sub_off_host, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(((uintptr_t)d_out & 3) == 0, LM_ERR_INVALID_ARG, "d_out must be 4-byte aligned");
    LM_CHECK(ev->n >= 0 && (ev->n == 0 || (ev->det1 && ev->det2)), LM_ERR_INVALID_ARG, "event detectors NULL");
    LM_CHECK(tof->n_bins == 0 || ev->n == 0 || ev->tof, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    const size_t need = sino_ws_layout(sc, n_subsets, nullptr, nullptr);
    LM_CHECK(ws != nullptr && ws_bytes >= need, LM_ERR_NOMEM, "sinogram counting needs %zu workspace bytes", need);
    SinoWs W;
    sino_ws_layout(sc, n_subsets, &W, ws);
    const int n_xtal = sc->n_xtal;
    const int64_t np = (int64_t)n_xtal * (n_xtal - 1) / 2;
    const int nb = std::max(1, (int)tof->n_bins);
    const int64_t per_q = (int64_t)sc->n_rings * sc->n_rings * nb;
    std::vector<int> qsub, qrank;
    std::vector<int32_t> qlist;
    std::vector<int64_t> qoff;
    view_tables(n_xtal, n_subsets, per_q, qsub, qrank, qlist, qoff, sub_off_host);
    const int64_t total = np * per_q;
    cudaStream_t st = S(stream);
    LM_CUDA(cudaMemcpyAsync(W.qsub, qsub.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(W.qrank, qrank.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(W.off, sub_off_host, (size_t)(n_subsets + 1) * 8, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(q_out, qlist.data(), (size_t)np * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(qoff_out, qoff.data(), (size_t)(n_subsets + 1) * 8, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemsetAsync(d_out, 0, (size_t)((total + 1) & ~(int64_t)1) * 2, st));
    LM_CUDA(cudaMemsetAsync(W.bad, 0, 4, st));
    if (ev->n > 0) {
        const int grid = (int)std::min<int64_t>((ev->n + 255) / 256, (int64_t)num_sms() * 16);
        sino_count_kernel<<<std::max(grid, 1), 256, 0, st>>>(n_xtal, sc->n_rings, nb, (nb - 1) / 2, ev->det1, ev->det2,
                                                             tof->n_bins > 0 ? ev->tof : nullptr, ev->n, W.qsub,
                                                             W.qrank, W.off, d_out, W.bad);
        count_launch();
        LM_CUDA(cudaGetLastError());
    }
    unsigned bad = 0;
    LM_CUDA(cudaMemcpyAsync(&bad, W.bad, 4, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(!(bad & 1u), LM_ERR_OUT_OF_RANGE, "an event has a detector or TOF bin out of range");
    LM_CHECK(!(bad & 2u), LM_ERR_OUT_OF_RANGE, "a sinogram bin holds more than 65535 events");
    return LM_OK;
}

}  // extern "C"
