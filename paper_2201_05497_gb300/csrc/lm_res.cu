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

// ---- fused passes: the x and y passes of one z slice in one block, then
// the z pass (with the layouts the caller needs) in a second kernel.  Each
// output is the same chain of fused multiply-adds over the same inputs as
// in res_row_kernel and res_march_kernel, so the results are identical.
constexpr int RT_X = 32, RT_Y = 32, RZ_SEG = 8;

// Input of the x and y passes at voxel (gx, gy) of slice z: the image, or
// (fold) the back-projection accumulators folded as res_fold_kernel does
// (std part; the y-fastest part is added by the caller).
__device__ __forceinline__ float res_in_std(const float* __restrict__ src, const float* __restrict__ acc_std,
                                            int64_t j, int64_t sz, bool below)
{
    if (acc_std == nullptr) return __ldg(src + j);
    return __ldg(acc_std + 2 * j) + (below ? __ldg(acc_std + 2 * (j - sz) + 1) : 0.0f);
}

// Loads of the x/y pass's input tile of slice z (thread tid's share, NL
// values): the std part into vs and, for the fold, the y-fastest part into vy.
template <int R, int NL>
__device__ __forceinline__ void res_xy_load(const float* __restrict__ src, const float* __restrict__ acc_std,
                                            const float* __restrict__ acc_yf, int nx, int ny, int x0, int y0, int z,
                                            int tid, float* vs, float* vy)
{
    constexpr int W = RT_X + 2 * R, H = RT_Y + 2 * R;
    const int64_t sz = (int64_t)nx * ny;
    const bool below = z > 0;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        const int i = tid + 256 * q;
        const int ly = i / W, lx = i - ly * W;
        const int gx = x0 - R + lx, gy = y0 - R + ly;
        vs[q] = 0.0f;
        if (i < H * W && gx <= nx - 1 + R && gy <= ny - 1 + R)
            vs[q] = res_in_std(src, acc_std, (int64_t)z * sz + (int64_t)mirror(gy, ny) * nx + mirror(gx, nx), sz,
                               below);
    }
    if (acc_yf != nullptr) {
        // the y-fastest accumulators, read along y (coalesced)
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int i = tid + 256 * q;
            const int lx = i / H, ly = i - lx * H;
            const int gx = x0 - R + lx, gy = y0 - R + ly;
            vy[q] = 0.0f;
            if (i < H * W && gx <= nx - 1 + R && gy <= ny - 1 + R) {
                const int64_t k = ((int64_t)z * nx + mirror(gx, nx)) * ny + mirror(gy, ny);
                vy[q] = __ldg(acc_yf + 2 * k) + (below ? __ldg(acc_yf + 2 * (k - sz) + 1) : 0.0f);
            }
        }
    }
}

// x pass then y pass of a RT_X x RT_Y tile of slice blockIdx.z, from the
// (RT_X + 2R) x (RT_Y + 2R) mirrored inputs around it staged in shared
// memory; every thread issues all of its loads before the first store (one
// tile per block: on the 200 x 200 x 96 grid this beat a resident grid
// looping over the tiles, with or without the next tile's loads in flight).
// Input: src, or with acc_std set the folded accumulators (read, not
// cleared: neighbouring tiles read them as halo).  Output: dst (x-fastest),
// or pairs (value, 0) when pair_out.
template <int R>
__global__ void __launch_bounds__(256) res_xy_kernel(const float* __restrict__ src, const float* __restrict__ acc_std,
                                                     const float* __restrict__ acc_yf, float* __restrict__ dst, int nx,
                                                     int ny, lmh::ResAxis wx, lmh::ResAxis wy, const uint16_t* seq,
                                                     int u, int n_subsets, int pair_out)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;
    constexpr int W = RT_X + 2 * R, H = RT_Y + 2 * R, NL = (H * W + 255) / 256;
    __shared__ float s_in[H][W + 1];
    __shared__ float s_x[H][RT_X + 1];
    const int x0 = blockIdx.x * RT_X, y0 = blockIdx.y * RT_Y, z = blockIdx.z;
    const int tid = threadIdx.x;
    const int64_t sz = (int64_t)nx * ny;
    float vs[NL], vy[NL];
    res_xy_load<R, NL>(src, acc_std, acc_yf, nx, ny, x0, y0, z, tid, vs, vy);
    const bool fold_std_only = acc_std != nullptr && acc_yf == nullptr;
#pragma unroll
    for (int q = 0; q < NL; ++q) {
        const int i = tid + 256 * q;
        const int ly = i / W, lx = i - ly * W;
        // (as the fold without y-fastest accumulators: the std part plus 0)
        if (i < H * W) s_in[ly][lx] = fold_std_only ? vs[q] + 0.0f : vs[q];
    }
    if (acc_yf != nullptr) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int i = tid + 256 * q;
            const int lx = i / H, ly = i - lx * H;
            if (i < H * W) s_in[ly][lx] = s_in[ly][lx] + vy[q];
        }
    }
    __syncthreads();
    for (int i = tid; i < H * RT_X; i += 256) {
        const int ly = i / RT_X, ox = i - ly * RT_X;
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wx.w[k], s_in[ly][ox + k], acc);
        s_x[ly][ox] = acc;
    }
    __syncthreads();
    for (int i = tid; i < RT_X * RT_Y; i += 256) {
        const int oy = i / RT_X, ox = i - oy * RT_X;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx < nx && gy < ny) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wy.w[k], s_x[oy + k][ox], acc);
            const int64_t j = (int64_t)z * sz + (int64_t)gy * nx + gx;
            if (pair_out)
                reinterpret_cast<float2*>(dst)[j] = make_float2(acc, 0.0f);
            else
                dst[j] = acc;
        }
    }
}

// z pass of a RT_X x RZ_Y column tile over RZ_SEG slices (one item per
// block): each thread loads the RZ_SEG + 2R inputs of each of its two
// columns into registers at once, then forms the columns' outputs from
// them.  Outputs: dst (x-fastest, or pairs (value, 0) when pair_out), dst_yf
// (y-fastest copy through a shared-memory transpose, or NULL); clear
// (n_clear floats, 16-byte aligned) is zeroed by the blocks together (the
// y-fastest accumulators, already folded by res_xy_kernel).
constexpr int RZ_Y = 16, RZ_CQ = RZ_Y / 8;

template <int R>
__global__ void __launch_bounds__(256) res_z_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                    float* __restrict__ dst_yf, float* __restrict__ clear,
                                                    int64_t n_clear, int nx, int ny, int nz, lmh::ResAxis wz,
                                                    const uint16_t* seq, int u, int n_subsets, int pair_out)
{
    if (seq != nullptr && seq[u] >= n_subsets) return;
    __shared__ float s_t[RZ_Y][RT_X + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x0 = blockIdx.x * RT_X, y0 = blockIdx.y * RZ_Y;
    const int64_t sz = (int64_t)nx * ny;
    if (clear != nullptr) {
        // this block's share of the n_clear floats: a range of whole float4s
        const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int64_t per = ((n_clear + nb - 1) / nb + 3) & ~(int64_t)3;
        const int64_t e0 = min(n_clear, b * per), e1 = min(n_clear, e0 + per);
        for (int64_t q = (e0 >> 2) + threadIdx.x; q < (e1 >> 2); q += 256)
            reinterpret_cast<float4*>(clear)[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int64_t i = (e1 & ~(int64_t)3) + threadIdx.x; i < e1; i += 256)
            if (i >= e0) clear[i] = 0.0f;
    }
    const int c0 = blockIdx.z * RZ_SEG;
    const int c1 = min(nz, c0 + RZ_SEG);
    constexpr int NV = RZ_SEG + 2 * R;  // inputs of a column's RZ_SEG outputs
    float wr[2 * R + 1];
#pragma unroll
    for (int k = 0; k <= 2 * R; ++k) wr[k] = wz.w[k];
    const int gx = x0 + tx;
    bool ok[RZ_CQ];
    int64_t base[RZ_CQ];
    float v[RZ_CQ][NV];
#pragma unroll
    for (int q = 0; q < RZ_CQ; ++q) {
        const int gy = y0 + ty + 8 * q;
        ok[q] = gx < nx && gy < ny;
        base[q] = (int64_t)gy * nx + gx;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const int c = c0 - R + k;
            v[q][k] = (ok[q] && c <= nz - 1 + R) ? __ldg(src + base[q] + (int64_t)mirror(c, nz) * sz) : 0.0f;
        }
    }
    // the y-fastest copy: value i = threadIdx.x + 256 q of a slice is (x = i / RZ_Y, y = i % RZ_Y), so
    // the lanes write runs of RZ_Y consecutive y
#pragma unroll
    for (int cc = 0; cc < RZ_SEG; ++cc) {
        const int c = c0 + cc;
        if (c >= c1) break;  // the same for the whole block
#pragma unroll
        for (int q = 0; q < RZ_CQ; ++q) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * R; ++k) acc = fmaf(wr[k], v[q][cc + k], acc);
            const int64_t j = (int64_t)c * sz + base[q];
            if (ok[q]) {
                if (pair_out)
                    reinterpret_cast<float2*>(dst)[j] = make_float2(acc, 0.0f);
                else
                    dst[j] = acc;
            }
            if (dst_yf != nullptr) s_t[ty + 8 * q][tx] = acc;
        }
        if (dst_yf != nullptr) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < RZ_CQ; ++q) {
                const int i = threadIdx.x + 256 * q;
                const int lx = i / RZ_Y, ly = i % RZ_Y;
                const int xx = x0 + lx, yy = y0 + ly;
                if (xx < nx && yy < ny) dst_yf[((int64_t)c * nx + xx) * ny + yy] = s_t[ly][lx];
            }
            __syncthreads();
        }
    }
}

}  // namespace

namespace lmh {

// Whether the fused passes serve plan p: x, y (and z) with one radius on x
// and y of at most 8 taps per side (and at most 8 on z).
static int fused_kind(const lm_grid* g, const ResPlan& p)
{
    if (p.n_axes < 2 || p.axis[0] != 0 || p.axis[1] != 1) return 0;
    const int r = p.ax[0].r;
    if (r < 1 || r > 8 || p.ax[1].r != r) return 0;
    if (p.n_axes == 2) return g->n[2] == 1 ? 2 : 0;
    if (p.axis[2] != 2 || p.ax[2].r < 1 || p.ax[2].r > 8 || g->n[2] > 65535) return 0;
    return 3;
}

template <int R>
static void launch_xy_r(const lm_grid* g, const ResPlan& p, const float* src, const float* acc_std,
                        const float* acc_yf, float* dst, const uint16_t* seq, int u, int n_subsets, cudaStream_t st,
                        bool pair_out)
{
    const dim3 grid((g->n[0] + RT_X - 1) / RT_X, (g->n[1] + RT_Y - 1) / RT_Y, g->n[2]);
    res_xy_kernel<R><<<grid, 256, 0, st>>>(src, acc_std, acc_yf, dst, g->n[0], g->n[1], p.ax[0], p.ax[1], seq, u,
                                           n_subsets, pair_out ? 1 : 0);
}

static void launch_xy(const lm_grid* g, const ResPlan& p, const float* src, const float* acc_std,
                      const float* acc_yf, float* dst, const uint16_t* seq, int u, int n_subsets, cudaStream_t st,
                      bool pair_out)
{
    switch (p.ax[0].r) {
        case 1: launch_xy_r<1>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 2: launch_xy_r<2>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 3: launch_xy_r<3>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 4: launch_xy_r<4>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 5: launch_xy_r<5>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 6: launch_xy_r<6>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        case 7: launch_xy_r<7>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
        default: launch_xy_r<8>(g, p, src, acc_std, acc_yf, dst, seq, u, n_subsets, st, pair_out); break;
    }
    count_launch();
}

template <int R>
static void launch_z_r(const lm_grid* g, const ResPlan& p, const float* src, float* dst, float* dst_yf, float* clear,
                       int64_t n_clear, const uint16_t* seq, int u, int n_subsets, cudaStream_t st, bool pair_out)
{
    const dim3 grid((g->n[0] + RT_X - 1) / RT_X, (g->n[1] + RZ_Y - 1) / RZ_Y, (g->n[2] + RZ_SEG - 1) / RZ_SEG);
    res_z_kernel<R><<<grid, 256, 0, st>>>(src, dst, dst_yf, clear, n_clear, g->n[0], g->n[1], g->n[2], p.ax[2], seq,
                                          u, n_subsets, pair_out ? 1 : 0);
}

static void launch_z(const lm_grid* g, const ResPlan& p, const float* src, float* dst, float* dst_yf, float* clear,
                     int64_t n_clear, const uint16_t* seq, int u, int n_subsets, cudaStream_t st, bool pair_out)
{
    switch (p.ax[2].r) {
        case 1: launch_z_r<1>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 2: launch_z_r<2>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 3: launch_z_r<3>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 4: launch_z_r<4>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 5: launch_z_r<5>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 6: launch_z_r<6>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        case 7: launch_z_r<7>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
        default: launch_z_r<8>(g, p, src, dst, dst_yf, clear, n_clear, seq, u, n_subsets, st, pair_out); break;
    }
    count_launch();
}

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
               const uint16_t* seq, int u, int n_subsets, cudaStream_t st, bool pair_out, float* dst_yf)
{
    const int V = (int)nvox(g);
    const dim3 blocks = res_grid(g);
    const int k = p.n_axes;
    if (k == 0) {
        if (src != dst) LM_CUDA(cudaMemcpyAsync(dst, src, (size_t)V * 4, cudaMemcpyDeviceToDevice, st));
        if (dst_yf != nullptr) launch_transpose_to_yf(g, dst, dst_yf, st);
        return LM_OK;
    }
    const int fk = fused_kind(g, p);
    if (fk == 3) {
        // x and y passes into t1, then the z pass into dst (and the y-fastest copy)
        launch_xy(g, p, src, nullptr, nullptr, t1, seq, u, n_subsets, st, false);
        launch_z(g, p, t1, dst, dst_yf, nullptr, 0, seq, u, n_subsets, st, pair_out);
        LM_CUDA(cudaGetLastError());
        return LM_OK;
    }
    if (fk == 2 && src != dst) {
        launch_xy(g, p, src, nullptr, nullptr, dst, seq, u, n_subsets, st, pair_out);
        if (dst_yf != nullptr) launch_transpose_to_yf(g, dst, dst_yf, st);
        LM_CUDA(cudaGetLastError());
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
    if (dst_yf != nullptr) launch_transpose_to_yf(g, dst, dst_yf, st);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int launch_res_back(const lm_grid* g, const ResPlan& p, float* acc_std, float* acc_yf, float* s1, float* s2,
                    const uint16_t* seq, int u, int n_subsets, cudaStream_t st)
{
    if (fused_kind(g, p) == 3) {
        // fold inside the x/y passes (the accumulators are read as halo by neighbouring
        // tiles, so they are cleared afterwards): the z pass writes every std pair as
        // (G A^T v, 0) and zeroes the y-fastest pairs
        launch_xy(g, p, nullptr, acc_std, acc_yf, s1, seq, u, n_subsets, st, false);
        launch_z(g, p, s1, acc_std, nullptr, acc_yf, acc_yf ? 2 * nvox(g) : 0, seq, u, n_subsets, st, true);
        LM_CUDA(cudaGetLastError());
        return LM_OK;
    }
    launch_res_fold(g, acc_std, acc_yf, s2, seq, u, n_subsets, st);
    return launch_res(g, p, s2, acc_std, s1, s2, seq, u, n_subsets, st, true, nullptr);
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
    return lmh::launch_res(grid, p, x, out, t1, t2, nullptr, 0, 0, lmh::S(stream), false, nullptr);
}

}  // extern "C"
