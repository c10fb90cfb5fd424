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
                                                       const uint16_t* seq, int u, int n_subsets, int pair_out)
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
    // pair_out: the first half of voxel j's (j, j + nx*ny) accumulator pair
    dst[pair_out ? 2 * (int64_t)j : j] = acc;
}

// The back-projection accumulators as one image: voxel j is the first half of
// its own std pair plus the second half of the pair below, plus the same from
// the y-fastest pairs (read through a shared-memory transpose); every half is
// cleared by its reader, as in the image pass.
constexpr int FT = 32, FR = 8;
__global__ void __launch_bounds__(256) res_fold_kernel(float* __restrict__ acc_std, float* __restrict__ acc_yf,
                                                       float* __restrict__ out, int nx, int ny, int nz,
                                                       const uint16_t* seq, int u, int n_subsets)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;
    __shared__ float sm[FT][FT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tiles_x = (nx + FT - 1) / FT, tiles_y = (ny + FT - 1) / FT;
    const int64_t sz = (int64_t)nx * ny;
    const int64_t n_tiles = (int64_t)tiles_x * tiles_y * nz;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int x0 = (int)(t % tiles_x) * FT;
        const int y0 = (int)((t / tiles_x) % tiles_y) * FT;
        const int z = (int)(t / ((int64_t)tiles_x * tiles_y));
        const bool below = z > 0;
        if (acc_yf != nullptr) {
            for (int r = ty; r < FT; r += FR) {
                const int xx = x0 + r, yy = y0 + tx;
                float v = 0.0f;
                if (xx < nx && yy < ny) {
                    const int64_t k = ((int64_t)z * nx + xx) * ny + yy;
                    v = acc_yf[2 * k] + (below ? acc_yf[2 * (k - sz) + 1] : 0.0f);
                    acc_yf[2 * k] = 0.0f;
                    if (below) acc_yf[2 * (k - sz) + 1] = 0.0f;
                }
                sm[r][tx] = v;
            }
        }
        __syncthreads();
        for (int r = ty; r < FT; r += FR) {
            const int xx = x0 + tx, yy = y0 + r;
            if (xx < nx && yy < ny) {
                const int64_t j = ((int64_t)z * ny + yy) * nx + xx;
                float v = acc_std[2 * j] + (below ? acc_std[2 * (j - sz) + 1] : 0.0f);
                if (acc_yf != nullptr) v += sm[tx][r];
                acc_std[2 * j] = 0.0f;
                if (below) acc_std[2 * (j - sz) + 1] = 0.0f;
                out[j] = v;
            }
        }
        __syncthreads();
    }
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

// dst = G src through the temporaries t1, t2 (pass i > 0 reads the previous
// pass's output, so t2 may be src; dst must alias neither t1 nor t2 unless it
// is src with one pass).  pair_out: dst is a pair accumulator (first halves).
// With seq set, nothing runs when seq[u] selects the prior.
int launch_res(const lm_grid* g, const ResPlan& p, const float* src, float* dst, float* t1, float* t2,
               const uint16_t* seq, int u, int n_subsets, cudaStream_t st, bool pair_out)
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
        const bool last = i == k - 1;
        float* out = last ? (in == dst ? t2 : dst) : ((i & 1) ? t2 : t1);
        res_pass_kernel<<<blocks, 256, 0, st>>>(in, out, g->n[0], g->n[1], g->n[2], p.axis[i], p.ax[i], seq, u,
                                                n_subsets, (last && out == dst && pair_out) ? 1 : 0);
        in = out;
    }
    count_launch(k);
    if (in != dst) {
        // one pass in place: copy the result back (skipped like the pass for a prior update)
        res_pass_kernel<<<blocks, 256, 0, st>>>(in, dst, g->n[0], g->n[1], g->n[2], 0, ResAxis{0, {1.0f}}, seq, u,
                                                n_subsets, pair_out ? 1 : 0);
        count_launch();
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

void launch_res_fold(const lm_grid* g, float* acc_std, float* acc_yf, float* out, const uint16_t* seq, int u,
                     int n_subsets, cudaStream_t st)
{
    const int64_t tiles = (int64_t)((g->n[0] + FT - 1) / FT) * ((g->n[1] + FT - 1) / FT) * g->n[2];
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 8);
    res_fold_kernel<<<std::max(grid, 1), dim3(FT, FR), 0, st>>>(acc_std, g->n[1] > 1 ? acc_yf : nullptr, out, g->n[0],
                                                               g->n[1], g->n[2], seq, u, n_subsets);
    count_launch();
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
    return lmh::launch_res(grid, p, x, out, t1, t2, nullptr, 0, 0, lmh::S(stream), false);
}

}  // extern "C"
