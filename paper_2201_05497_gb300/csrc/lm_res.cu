// Image-space resolution model of the forward model P = A G (Eq. (1): P
// includes the scanner's limited spatial resolution).  G is a separable
// Gaussian blur of full width at half maximum fwhm (mm) on every axis with
// more than one voxel: sigma_d = fwhm / (2 sqrt(2 ln 2)) / h_d voxels, taps
// k = -r..r with r = floor(3 sigma_d + 1/2) (at most n_d - 1), weights
// exp(-k^2 / (2 sigma_d^2)) normalised to sum 1, and the image mirrored about
// its outer faces (index -1 reads 0, index n reads n - 1).  This G is
// symmetric and its rows sum to 1, so P^T = G A^T and P 1 = A 1.
//
// One pass per axis; a thread computes one output voxel from the 2r + 1
// inputs along the axis (consecutive threads take consecutive x, so every
// tap's loads are coalesced and neighbouring outputs share them in L1/L2).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lm_internal.h"

namespace {

__global__ void __launch_bounds__(256) res_pass_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                       int nx, int ny, int nz, int axis, lmh::ResAxis w,
                                                       const uint16_t* seq, int u, int n_subsets)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;  // a prior update back-projects nothing
    const int V = nx * ny * nz;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= V) return;
    int c, n, st;
    if (axis == 0) {
        c = j % nx;
        n = nx;
        st = 1;
    } else if (axis == 1) {
        c = (j / nx) % ny;
        n = ny;
        st = nx;
    } else {
        c = j / (nx * ny);
        n = nz;
        st = nx * ny;
    }
    const int r = w.r;
    float acc = 0.0f;
    for (int k = -r; k <= r; ++k) {
        int m = c + k;
        if (m < 0) m = -m - 1;
        if (m >= n) m = 2 * n - m - 1;
        acc = fmaf(w.w[k + r], __ldg(src + j + (m - c) * st), acc);
    }
    dst[j] = acc;
}

}  // namespace

namespace lmh {

int res_plan(const lm_grid* g, float fwhm, ResPlan& p)
{
    std::memset(&p, 0, sizeof(p));
    if (!(fwhm > 0.0f)) return LM_OK;
    LM_CHECK(std::isfinite(fwhm), LM_ERR_INVALID_ARG, "resolution FWHM must be finite");
    for (int d = 0; d < 3; ++d) {
        const int n = g->n[d];
        if (n < 2) continue;
        const double sig = (double)fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0))) / (double)g->h[d];
        int r = (int)std::floor(3.0 * sig + 0.5);
        r = std::min(r, n - 1);
        LM_CHECK(r <= RES_MAX_R, LM_ERR_INVALID_ARG, "resolution kernel too wide: %d taps per side (at most %d)", r,
                 RES_MAX_R);
        ResAxis& a = p.ax[p.n_axes];
        a.r = r;
        double wd[2 * RES_MAX_R + 1];
        double sum = 0.0;
        for (int k = -r; k <= r; ++k) {
            wd[k + r] = std::exp(-(double)k * k / (2.0 * sig * sig));
            sum += wd[k + r];
        }
        for (int k = 0; k <= 2 * r; ++k) a.w[k] = (float)(wd[k] / sum);
        p.axis[p.n_axes] = d;
        ++p.n_axes;
    }
    return LM_OK;
}

// dst = G src through the temporaries t1, t2 (src may equal dst; neither may
// alias t1 or t2).  With seq set, nothing runs when seq[u] selects the prior.
int launch_res(const lm_grid* g, const ResPlan& p, const float* src, float* dst, float* t1, float* t2,
               const uint16_t* seq, int u, int n_subsets, cudaStream_t st)
{
    const int V = (int)nvox(g);
    const int blocks = (V + 255) / 256;
    const int k = p.n_axes;
    if (k == 0) {
        if (src != dst) LM_CUDA(cudaMemcpyAsync(dst, src, (size_t)V * 4, cudaMemcpyDeviceToDevice, st));
        return LM_OK;
    }
    const float* in = src;
    for (int i = 0; i < k; ++i) {
        float* out = (i == k - 1) ? (in == dst ? t2 : dst) : ((i & 1) ? t2 : t1);
        res_pass_kernel<<<blocks, 256, 0, st>>>(in, out, g->n[0], g->n[1], g->n[2], p.axis[i], p.ax[i], seq, u,
                                                n_subsets);
        in = out;
    }
    count_launch(k);
    if (in != dst) {
        // one pass in place: copy the result back (skipped like the pass for a prior update)
        res_pass_kernel<<<blocks, 256, 0, st>>>(in, dst, g->n[0], g->n[1], g->n[2], 0, ResAxis{0, {1.0f}}, seq, u,
                                                n_subsets);
        count_launch();
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

}  // namespace lmh

extern "C" {

size_t lm_res_workspace_bytes(const lm_grid* grid)
{
    if (lmh::check_grid(grid)) return 0;
    return 2 * lmh::align_up((size_t)lmh::nvox(grid) * 4);
}

int lm_res_apply(const lm_grid* grid, float fwhm, const float* x, float* out, void* ws, size_t ws_bytes,
                 void* stream)
{
    lmh::clear_error();
    int rc = lmh::check_grid(grid);
    if (rc) return rc;
    LM_CHECK(x && out, LM_ERR_INVALID_ARG, "x or out is NULL");
    LM_CHECK(fwhm >= 0.0f, LM_ERR_INVALID_ARG, "fwhm must be >= 0");
    LM_CHECK(ws != nullptr && ws_bytes >= lm_res_workspace_bytes(grid), LM_ERR_NOMEM,
             "the resolution model needs %zu workspace bytes", lm_res_workspace_bytes(grid));
    lmh::ResPlan p;
    rc = lmh::res_plan(grid, fwhm, p);
    if (rc) return rc;
    float* t1 = (float*)ws;
    float* t2 = (float*)((char*)ws + lmh::align_up((size_t)lmh::nvox(grid) * 4));
    return lmh::launch_res(grid, p, x, out, t1, t2, nullptr, 0, 0, lmh::S(stream));
}

}  // extern "C"
