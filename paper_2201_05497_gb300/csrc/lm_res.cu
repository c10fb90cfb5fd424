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
// Blocks cover row segments (grid.x along x, grid.y the (y, z) rows), so no
// thread divides its voxel index; taps mirror only near the faces.
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
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    if (ix >= nx) return;
    const int row = blockIdx.y + gridDim.y * blockIdx.z;  // row = iz * ny + iy
    if (row >= ny * nz) return;
    const int j = row * nx + ix;
    int c, n, st;
    if (axis == 0) {
        c = ix;
        n = nx;
        st = 1;
    } else if (axis == 1) {
        c = row % ny;
        n = ny;
        st = nx;
    } else {
        c = row / ny;
        n = nz;
        st = nx * ny;
    }
    const int r = w.r;
    const float* s0 = src + j;
    float acc = 0.0f;
    if (c >= r && c + r < n) {
        for (int k = -r; k <= r; ++k) acc = fmaf(w.w[k + r], __ldg(s0 + k * st), acc);
    } else {
        for (int k = -r; k <= r; ++k) {
            int m = c + k;
            if (m < 0) m = -m - 1;
            if (m >= n) m = 2 * n - m - 1;
            acc = fmaf(w.w[k + r], __ldg(s0 + (m - c) * st), acc);
        }
    }
    // pair_out: the first half of voxel j's (j, j + nx*ny) accumulator pair
    dst[pair_out ? 2 * (int64_t)j : j] = acc;
}

// The y and z passes with up to 8 taps per side march along their axis: a
// thread owns one x of one line and a segment of RES_SEG outputs, keeps the
// 2R + 1 inputs of the current output in registers and loads each input
// once (the window's first 2R on entry).  Same products in the same order as
// res_pass_kernel, so the results are identical.
constexpr int RES_SEG = 16;

__device__ __forceinline__ int mirror(int m, int n) { return m < 0 ? -m - 1 : (m >= n ? 2 * n - m - 1 : m); }

template <int R>
__global__ void __launch_bounds__(256) res_march_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                        int nx, int ny, int nz, int axis, lmh::ResAxis w,
                                                        const uint16_t* seq, int u, int n_subsets, int pair_out)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    if (ix >= nx) return;
    const int o = blockIdx.y;  // z of a y line, y of a z line
    int n, st, base;
    if (axis == 1) {
        n = ny;
        st = nx;
        base = o * nx * ny + ix;
    } else {
        n = nz;
        st = nx * ny;
        base = o * nx + ix;
    }
    const int c0 = blockIdx.z * RES_SEG;
    if (c0 >= n) return;
    const int c1 = min(n, c0 + RES_SEG);
    float wr[2 * R + 1], v[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) wr[k] = w.w[k];
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) v[k + 1] = __ldg(src + base + mirror(c0 - R + k, n) * st);
    // unrolled so that several outputs' loads are in flight per thread
#pragma unroll 4
    for (int c = c0; c < c1; ++c) {
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) v[k] = v[k + 1];
        v[2 * R] = __ldg(src + base + mirror(c + R, n) * st);
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wr[k], v[k], acc);
        const int64_t j = (int64_t)base + (int64_t)c * st;
        dst[pair_out ? 2 * j : j] = acc;
    }
}

// The x pass with up to 8 taps per side: taps unrolled with the weights and
// the (mirrored) tap offsets in registers, RES_ROWS rows per thread so that
// their loads are in flight together.  Same products in the same order as
// res_pass_kernel, so the results are identical.
constexpr int RES_ROWS = 4;

template <int R>
__global__ void __launch_bounds__(256) res_row_kernel(const float* __restrict__ src, float* __restrict__ dst, int nx,
                                                      int rows, lmh::ResAxis w, const uint16_t* seq, int u,
                                                      int n_subsets, int pair_out)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    if (ix >= nx) return;
    const int row0 = (blockIdx.y + gridDim.y * blockIdx.z) * RES_ROWS;
    if (row0 >= rows) return;
    float wr[2 * R + 1];
    int off[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) {
        wr[k] = w.w[k];
        off[k] = mirror(ix - R + k, nx) - ix;
    }
    float acc[RES_ROWS];
#pragma unroll
    for (int q = 0; q < RES_ROWS; ++q) {
        acc[q] = 0.0f;
        if (row0 + q < rows) {
            const float* s0 = src + (int64_t)(row0 + q) * nx + ix;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) acc[q] = fmaf(wr[k], __ldg(s0 + off[k]), acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < RES_ROWS; ++q) {
        if (row0 + q < rows) {
            const int64_t j = (int64_t)(row0 + q) * nx + ix;
            dst[pair_out ? 2 * j : j] = acc[q];
        }
    }
}

// Threads per block: a whole row rounded up to a warp, at most 256.
int res_block(const lm_grid* g) { return std::min(256, (g->n[0] + 31) / 32 * 32); }

dim3 res_grid(const lm_grid* g)
{
    const int rows = g->n[1] * g->n[2];
    const int gy = std::min(rows, 65535);
    const int bx = res_block(g);
    return dim3((g->n[0] + bx - 1) / bx, gy, (rows + gy - 1) / gy);
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
        // all loads of the thread's rows first (memory-level parallelism), then the clears
        constexpr int RPT = FT / FR;
        if (acc_yf != nullptr) {
            float v[RPT];
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int xx = x0 + ty + q * FR, yy = y0 + tx;
                v[q] = 0.0f;
                if (xx < nx && yy < ny) {
                    const int64_t k = ((int64_t)z * nx + xx) * ny + yy;
                    v[q] = acc_yf[2 * k] + (below ? acc_yf[2 * (k - sz) + 1] : 0.0f);
                }
            }
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int xx = x0 + ty + q * FR, yy = y0 + tx;
                if (xx < nx && yy < ny) {
                    const int64_t k = ((int64_t)z * nx + xx) * ny + yy;
                    acc_yf[2 * k] = 0.0f;
                    if (below) acc_yf[2 * (k - sz) + 1] = 0.0f;
                }
                sm[ty + q * FR][tx] = v[q];
            }
        }
        __syncthreads();
        float v[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int xx = x0 + tx, yy = y0 + ty + q * FR;
            v[q] = 0.0f;
            if (xx < nx && yy < ny) {
                const int64_t j = ((int64_t)z * ny + yy) * nx + xx;
                v[q] = acc_std[2 * j] + (below ? acc_std[2 * (j - sz) + 1] : 0.0f);
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = ty + q * FR;
            const int xx = x0 + tx, yy = y0 + r;
            if (xx < nx && yy < ny) {
                const int64_t j = ((int64_t)z * ny + yy) * nx + xx;
                acc_std[2 * j] = 0.0f;
                if (below) acc_std[2 * (j - sz) + 1] = 0.0f;
                out[j] = v[q] + (acc_yf != nullptr ? sm[tx][r] : 0.0f);
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
    const dim3 blocks = res_grid(g);
    const int k = p.n_axes;
    if (k == 0) {
        if (src != dst) LM_CUDA(cudaMemcpyAsync(dst, src, (size_t)V * 4, cudaMemcpyDeviceToDevice, st));
        return LM_OK;
    }
    const float* in = src;
    for (int i = 0; i < k; ++i) {
        const bool last = i == k - 1;
        float* out = last ? (in == dst ? t2 : dst) : ((i & 1) ? t2 : t1);
        const int po = (last && out == dst && pair_out) ? 1 : 0;
        const int ax = p.axis[i], r = p.ax[i].r;
        const int lines = ax == 1 ? g->n[2] : g->n[1];
        if (ax == 0 && r >= 1 && r <= 8) {
            const int rows = g->n[1] * g->n[2];
            const int groups = (rows + RES_ROWS - 1) / RES_ROWS;
            const int gy = std::min(groups, 65535);
            const dim3 rg((g->n[0] + res_block(g) - 1) / res_block(g), gy, (groups + gy - 1) / gy);
#define LM_ROW(RR)                                                                                             \
    case RR:                                                                                                   \
        res_row_kernel<RR><<<rg, res_block(g), 0, st>>>(in, out, g->n[0], rows, p.ax[i], seq, u, n_subsets, po); \
        break;
            switch (r) {
                LM_ROW(1) LM_ROW(2) LM_ROW(3) LM_ROW(4) LM_ROW(5) LM_ROW(6) LM_ROW(7) LM_ROW(8)
            }
#undef LM_ROW
        } else if (ax > 0 && r >= 1 && r <= 8 && lines <= 65535) {
            const int n = g->n[ax];
            const dim3 mg((g->n[0] + res_block(g) - 1) / res_block(g), lines, (n + RES_SEG - 1) / RES_SEG);
#define LM_MARCH(RR)                                                                                             \
    case RR:                                                                                                     \
        res_march_kernel<RR><<<mg, res_block(g), 0, st>>>(in, out, g->n[0], g->n[1], g->n[2], ax, p.ax[i], seq, u, \
                                                          n_subsets, po);                                        \
        break;
            switch (r) {
                LM_MARCH(1) LM_MARCH(2) LM_MARCH(3) LM_MARCH(4) LM_MARCH(5) LM_MARCH(6) LM_MARCH(7) LM_MARCH(8)
            }
#undef LM_MARCH
        } else {
            res_pass_kernel<<<blocks, res_block(g), 0, st>>>(in, out, g->n[0], g->n[1], g->n[2], ax, p.ax[i], seq, u,
                                                             n_subsets, po);
        }
        in = out;
    }
    count_launch(k);
    if (in != dst) {
        // one pass in place: copy the result back (skipped like the pass for a prior update)
        res_pass_kernel<<<blocks, res_block(g), 0, st>>>(in, dst, g->n[0], g->n[1], g->n[2], 0, ResAxis{0, {1.0f}}, seq,
                                                         u, n_subsets, pair_out ? 1 : 0);
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
