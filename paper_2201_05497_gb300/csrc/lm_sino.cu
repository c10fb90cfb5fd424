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
    std::vector<int> qsub((size_t)np), qrank((size_t)np);
    std::vector<int64_t> cnt((size_t)n_subsets, 0);
    for (int64_t q = 0; q < np; ++q) {
        int c1, c2;
        pair_of_q(q, n_xtal, c1, c2);
        const int k = ((c1 + c2) % n_xtal) % n_subsets;
        qsub[(size_t)q] = k;
        qrank[(size_t)q] = (int)cnt[(size_t)k]++;
    }
    sub_off_host[0] = 0;
    for (int k = 0; k < n_subsets; ++k) sub_off_host[k + 1] = sub_off_host[k] + cnt[(size_t)k] * per_q;
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

}  // extern "C"
