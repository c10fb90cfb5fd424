// Image-space kernels of LM-SPDHG (Alg. 2): the per-update image pass that
// merges the back-projected dual change into z (compensated float32
// summation), forms zbar = z + dz/p_i and applies the next primal step
// x <- proj_{>=0}(x - T zbar) (the primal step that opens the following
// update of Alg. 2); the
// TV operator K (forward differences, Neumann boundary), its adjoint and the
// prox of R^* (Sec. "Numerical experiments"); the FP64 power iteration for
// ||K||; the step sizes T (Eq. lm_stepsizes) and FP64 reductions of the
// objective (Eq. 1).
//
// Image passes work on 32 x 32 (x, y) tiles of one z slice so that the
// y-fastest copies are read and written through shared memory with
// coalesced accesses in both layouts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "lm_internal.h"

using namespace lmk;

namespace {

constexpr int TD = 32;  // tile edge
constexpr int TR = 8;   // thread rows per tile (block 32 x 8)

struct TileIdx {
    int x0, y0, z;
};

__device__ __forceinline__ TileIdx tile_of(int64_t t, int nx, int ny)
{
    const int tx = (nx + TD - 1) / TD, ty = (ny + TD - 1) / TD;
    TileIdx r;
    r.x0 = (int)(t % tx) * TD;
    r.y0 = (int)((t / tx) % ty) * TD;
    r.z = (int)(t / ((int64_t)tx * ty));
    return r;
}

__device__ __forceinline__ int64_t n_tiles(int nx, int ny, int nz)
{
    return (int64_t)((nx + TD - 1) / TD) * ((ny + TD - 1) / TD) * nz;
}

__global__ void __launch_bounds__(256) transpose_to_yf_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                              int nx, int ny, int nz)
{
    __shared__ float sm[TD][TD + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t t = blockIdx.x; t < n_tiles(nx, ny, nz); t += gridDim.x) {
        const TileIdx T = tile_of(t, nx, ny);
        for (int r = ty; r < TD; r += TR) {
            const int xx = T.x0 + tx, yy = T.y0 + r;
            if (xx < nx && yy < ny) sm[r][tx] = src[((int64_t)T.z * ny + yy) * nx + xx];
        }
        __syncthreads();
        for (int r = ty; r < TD; r += TR) {
            const int xx = T.x0 + r, yy = T.y0 + tx;
            if (xx < nx && yy < ny) dst[((int64_t)T.z * nx + xx) * ny + yy] = sm[tx][r];
        }
        __syncthreads();
    }
}

// img += transpose(yf); yf <- 0
__global__ void __launch_bounds__(256) add_yf_kernel(float* __restrict__ img, float* __restrict__ yf, int nx, int ny,
                                                     int nz)
{
    __shared__ float sm[TD][TD + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t t = blockIdx.x; t < n_tiles(nx, ny, nz); t += gridDim.x) {
        const TileIdx T = tile_of(t, nx, ny);
        for (int r = ty; r < TD; r += TR) {
            const int xx = T.x0 + r, yy = T.y0 + tx;
            if (xx < nx && yy < ny) {
                const int64_t k = ((int64_t)T.z * nx + xx) * ny + yy;
                sm[r][tx] = yf[k];
                yf[k] = 0.0f;
            }
        }
        __syncthreads();
        for (int r = ty; r < TD; r += TR) {
            const int xx = T.x0 + tx, yy = T.y0 + r;
            if (xx < nx && yy < ny) img[((int64_t)T.z * ny + yy) * nx + xx] += sm[tx][r];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double fx_step(const unsigned* maxbits, long long count, float stepmax)
{
    const float vmax = __uint_as_float(*maxbits);
    return ldexp(1.0, -fx_exponent(vmax, count, stepmax));
}

// img += (a_std + transpose(a_yf)) * 2^-E; accumulators <- 0
__global__ void __launch_bounds__(256) fold_fixed_kernel(float* __restrict__ img, unsigned long long* __restrict__ a_std,
                                                         unsigned long long* __restrict__ a_yf, const unsigned* maxbits,
                                                         long long count, float stepmax, int nx, int ny, int nz)
{
    __shared__ long long sm[TD][TD + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const double step = fx_step(maxbits, count, stepmax);
    for (int64_t t = blockIdx.x; t < n_tiles(nx, ny, nz); t += gridDim.x) {
        const TileIdx T = tile_of(t, nx, ny);
        if (a_yf) {
            for (int r = ty; r < TD; r += TR) {
                const int xx = T.x0 + r, yy = T.y0 + tx;
                if (xx < nx && yy < ny) {
                    const int64_t k = ((int64_t)T.z * nx + xx) * ny + yy;
                    sm[r][tx] = (long long)a_yf[k];
                    a_yf[k] = 0ULL;
                }
            }
        }
        __syncthreads();
        for (int r = ty; r < TD; r += TR) {
            const int xx = T.x0 + tx, yy = T.y0 + r;
            if (xx < nx && yy < ny) {
                const int64_t j = ((int64_t)T.z * ny + yy) * nx + xx;
                long long s = (long long)a_std[j];
                a_std[j] = 0ULL;
                if (a_yf) s += sm[tx][r];
                img[j] += (float)((double)s * step);
            }
        }
        __syncthreads();
    }
}

// Directional TV: (P d) at voxel m for d = w+ - w, P = I - xi xi^T of the
// voxel (components of axes of length 1 are 0).
__device__ __forceinline__ void dtv_pd(const lmh::ImgArgs& A, const float* wc, const float* wn, int64_t m, int cx,
                                       int cy, int cz, float& px, float& py, float& pz)
{
    const int64_t V = A.V;
    const float* f = A.xi;
    px = cx >= 0 ? wn[cx * V + m] - wc[cx * V + m] : 0.0f;
    py = cy >= 0 ? wn[cy * V + m] - wc[cy * V + m] : 0.0f;
    pz = cz >= 0 ? wn[cz * V + m] - wc[cz * V + m] : 0.0f;
    dtv_perp(cx >= 0 ? f[cx * V + m] : 0.0f, cy >= 0 ? f[cy * V + m] : 0.0f, cz >= 0 ? f[cz * V + m] : 0.0f, px, py,
             pz);
}

// dz_j = (K^T (w+ - w))_j = (grad^T P (w+ - w))_j for the directional TV
__device__ __noinline__ float prior_dz_dtv(const lmh::ImgArgs& A, const float* wc, const float* wn, int xx, int yy,
                                           int zz, int64_t j)
{
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    int c = 0;
    const int cx = nx > 1 ? c++ : -1;
    const int cy = ny > 1 ? c++ : -1;
    const int cz = nz > 1 ? c++ : -1;
    float px, py, pz, qx, qy, qz;
    dtv_pd(A, wc, wn, j, cx, cy, cz, px, py, pz);
    float dz = 0.0f;
    if (cx >= 0) {
        if (xx < nx - 1) dz -= px;
        if (xx >= 1) {
            dtv_pd(A, wc, wn, j - 1, cx, cy, cz, qx, qy, qz);
            dz += qx;
        }
    }
    if (cy >= 0) {
        if (yy < ny - 1) dz -= py;
        if (yy >= 1) {
            dtv_pd(A, wc, wn, j - nx, cx, cy, cz, qx, qy, qz);
            dz += qy;
        }
    }
    if (cz >= 0) {
        if (zz < nz - 1) dz -= pz;
        if (zz >= 1) {
            dtv_pd(A, wc, wn, j - (int64_t)nx * ny, cx, cy, cz, qx, qy, qz);
            dz += qz;
        }
    }
    return dz;
}

// dz_j = grad^T D at voxel j for D = P (w+ - w) stored by the directional
// TV's dual step (components in axis order; same sums as prior_dz_dtv)
__device__ __forceinline__ float prior_dz_dtv_stored(const lmh::ImgArgs& A, int xx, int yy, int zz, int64_t j)
{
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int64_t V = A.V;
    const float* D = A.dtv_d;
    float dz = 0.0f;
    int c = 0;
    if (nx > 1) {
        const int64_t o = (int64_t)c * V;
        if (xx < nx - 1) dz -= D[o + j];
        if (xx >= 1) dz += D[o + j - 1];
        ++c;
    }
    if (ny > 1) {
        const int64_t o = (int64_t)c * V;
        if (yy < ny - 1) dz -= D[o + j];
        if (yy >= 1) dz += D[o + j - nx];
        ++c;
    }
    if (nz > 1) {
        const int64_t o = (int64_t)c * V;
        if (zz < nz - 1) dz -= D[o + j];
        if (zz >= 1) dz += D[o + j - (int64_t)nx * ny];
    }
    return dz;
}

// dz_j = (K^T (w+ - w))_j, components in axis order for axes with n > 1
__device__ __forceinline__ float prior_dz(const lmh::ImgArgs& A, const float* wc, const float* wn, int xx, int yy,
                                          int zz, int64_t j)
{
    if (A.xi != nullptr)
        return A.dtv_d != nullptr ? prior_dz_dtv_stored(A, xx, yy, zz, j) : prior_dz_dtv(A, wc, wn, xx, yy, zz, j);
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int64_t V = A.V;
    float dz = 0.0f;
    int c = 0;
    if (nx > 1) {
        const int64_t o = (int64_t)c * V;
        if (xx < nx - 1) dz -= wn[o + j] - wc[o + j];
        if (xx >= 1) dz += wn[o + j - 1] - wc[o + j - 1];
        ++c;
    }
    if (ny > 1) {
        const int64_t o = (int64_t)c * V;
        if (yy < ny - 1) dz -= wn[o + j] - wc[o + j];
        if (yy >= 1) dz += wn[o + j - nx] - wc[o + j - nx];
        ++c;
    }
    if (nz > 1) {
        const int64_t o = (int64_t)c * V;
        const int64_t sz = (int64_t)nx * ny;
        if (zz < nz - 1) dz -= wn[o + j] - wc[o + j];
        if (zz >= 1) dz += wn[o + j - sz] - wc[o + j - sz];
    }
    return dz;
}

// What an image pass does at update u: merge the data accumulators (data
// update, or the initialisation) or form K^T(w+ - w) (prior update).
struct PassMode {
    bool data, prior, init;
    float inv_p;
    double fx;  // fixed-point step of the data accumulators (deterministic mode)
    const float* wc;
    const float* wn;
};

__device__ __forceinline__ PassMode pass_mode(const lmh::ImgArgs& A, int u)
{
    PassMode m;
    m.init = A.mode == lmh::IP_INIT;
    m.data = m.init;
    m.prior = false;
    m.inv_p = 1.0f;
    m.fx = 0.0;
    m.wc = m.wn = nullptr;
    long long count = 0;
    int slot = 1;  // max-bits slot of the fixed-point scale used by this update
    if (A.mode == lmh::IP_UPDATE) {
        const int sel = A.seq[u];
        m.prior = sel >= A.n_subsets;
        m.data = !m.prior;
        if (m.data) count = (long long)(A.sub_off[sel + 1] - A.sub_off[sel]);
        m.inv_p = m.prior ? A.inv_p_prior : A.inv_p_data;
        slot = (A.slot0 + u) & 1;
    } else {
        count = (long long)A.sub_off[A.n_subsets];
    }
    if (m.data && A.det) m.fx = fx_step(A.maxbits + slot, count, A.stepmax);
    if (m.prior) {
        const int wp = A.wpar[u];
        m.wc = A.w_cur[wp];
        m.wn = A.w_nxt[wp];
    }
    return m;
}

// Clears the fixed-point scale slot the next update will use (one thread).
__device__ __forceinline__ void reset_next_slot(const lmh::ImgArgs& A, int u)
{
    if (!A.maxbits_reset) return;
    if (A.mode == lmh::IP_UPDATE) A.maxbits_reset[(A.slot0 + u + 1) & 1] = 0u;
    else A.maxbits_reset[0] = 0u;
}

struct TileSmem {
    float f[TD][TD + 1];
    long long i[TD][TD + 1];
    float x[TD][TD + 1];
};

// One 32 x 32 tile of one z slice: all loads of the thread's rows first
// (memory-level parallelism), then compute and store; the y-fastest arrays
// go through shared memory so both layouts are accessed coalesced.
__device__ __forceinline__ void image_tile(const lmh::ImgArgs& A, const PassMode& m, int u, const TileIdx& Tl,
                                           const float* __restrict__ xcur, float* __restrict__ x_nxt_std,
                                           float* __restrict__ x_nxt_yf, TileSmem& sm)
{
    constexpr int RPT = TD / TR;  // rows per thread in a tile
    const int nx = A.n[0], ny = A.n[1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    // y-fastest accumulators and x copy (absent with the resolution model, whose projections read one layout)
    const bool have_yf = ny > 1 && (A.det ? A.acci_yf != nullptr : A.acc_yf != nullptr);
    const bool x_yf = ny > 1 && x_nxt_yf != nullptr;
    const bool kahan = A.kahan != 0;
    const bool det = A.det != 0;
    const float* __restrict__ Tm = A.T;
    float* __restrict__ zz = A.z;
    float* __restrict__ zc = A.zc;
    float* __restrict__ acc_std = A.acc_std;
    float* __restrict__ acc_yf = A.acc_yf;
    unsigned long long* __restrict__ acci_std = A.acci_std;
    unsigned long long* __restrict__ acci_yf = A.acci_yf;
    // float accumulators hold z pairs: voxel k is element 2k plus element
    // 2(k - nx*ny) + 1 of the slice below; each half is cleared by its reader
    const int64_t sz = (int64_t)nx * ny;
    const bool below = Tl.z > 0;
    if (m.data && have_yf) {
        float vf[RPT];
        long long vi[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = ty + q * TR;
            const int xx = Tl.x0 + r, yy = Tl.y0 + tx;
            vf[q] = 0.0f;
            vi[q] = 0;
            if (xx < nx && yy < ny) {
                const int64_t k = ((int64_t)Tl.z * nx + xx) * ny + yy;
                if (det) vi[q] = (long long)acci_yf[k];
                else if (A.acc_pairs) vf[q] = acc_yf[2 * k] + (below ? acc_yf[2 * (k - sz) + 1] : 0.0f);
                else vf[q] = acc_yf[k];
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = ty + q * TR;
            const int xx = Tl.x0 + r, yy = Tl.y0 + tx;
            if (xx < nx && yy < ny) {
                const int64_t k = ((int64_t)Tl.z * nx + xx) * ny + yy;
                if (det) {
                    sm.i[r][tx] = vi[q];
                    acci_yf[k] = 0ULL;
                } else {
                    sm.f[r][tx] = vf[q];
                    if (A.acc_pairs) {
                        acc_yf[2 * k] = 0.0f;
                        if (below) acc_yf[2 * (k - sz) + 1] = 0.0f;
                    } else {
                        acc_yf[k] = 0.0f;
                    }
                }
            }
        }
    }
    __syncthreads();
    float dz[RPT], x0[RPT], tm[RPT], z0[RPT], zl0[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int xx = Tl.x0 + tx, yy = Tl.y0 + ty + q * TR;
        dz[q] = x0[q] = tm[q] = z0[q] = zl0[q] = 0.0f;
        if (xx < nx && yy < ny) {
            const int64_t j = ((int64_t)Tl.z * ny + yy) * nx + xx;
            x0[q] = xcur[j];
            tm[q] = Tm[j];
            if (m.init) {
                z0[q] = A.sens[j];
            } else {
                z0[q] = zz[j];
                if (kahan) zl0[q] = zc[j];
            }
            if (m.data) {
                if (det) {
                    long long s = (long long)acci_std[j];
                    if (have_yf) s += sm.i[tx][ty + q * TR];
                    dz[q] = (float)((double)s * m.fx);
                } else {
                    dz[q] = A.acc_pairs ? acc_std[2 * j] + (below ? acc_std[2 * (j - sz) + 1] : 0.0f) : acc_std[j];
                    if (have_yf) dz[q] += sm.f[tx][ty + q * TR];
                }
            } else {
                dz[q] = prior_dz(A, m.wc, m.wn, xx, yy, Tl.z, j);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = ty + q * TR;
        const int xx = Tl.x0 + tx, yy = Tl.y0 + r;
        if (xx < nx && yy < ny) {
            const int64_t j = ((int64_t)Tl.z * ny + yy) * nx + xx;
            if (m.data) {
                if (det) {
                    acci_std[j] = 0ULL;
                } else if (A.acc_pairs) {
                    acc_std[2 * j] = 0.0f;
                    if (below) acc_std[2 * (j - sz) + 1] = 0.0f;
                } else {
                    acc_std[j] = 0.0f;
                }
            }
            float zh, zl = 0.0f, xn;
            if (m.init) {
                // z = P^T 1 + (P^LM)^T((y-1)/mu); zbar = z; first primal step from x0
                float e = 0.0f;
                two_sum(z0[q], dz[q], zh, e);
                zl = kahan ? e : 0.0f;
                A.x_keep[j] = x0[q];
                xn = fmaxf(0.0f, fmaf(-tm[q], zh + zl, x0[q]));
            } else {
                if (kahan) {
                    float e;
                    two_sum(z0[q], dz[q], zh, e);
                    zl = zl0[q] + e;
                } else {
                    zh = z0[q] + dz[q];
                }
                const float zbar = fmaf(dz[q], m.inv_p, zh + zl);  // z + dz/p_i
                xn = fmaxf(0.0f, fmaf(-tm[q], zbar, x0[q]));
            }
            zz[j] = zh;
            if (kahan) zc[j] = zl;
            x_nxt_std[j] = xn;
            sm.x[r][tx] = xn;
        }
    }
    __syncthreads();
    if (x_yf) {
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int r = ty + q * TR;
            const int xx = Tl.x0 + r, yy = Tl.y0 + tx;
            if (xx < nx && yy < ny) x_nxt_yf[((int64_t)Tl.z * nx + xx) * ny + yy] = sm.x[tx][r];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) image_pass_kernel(const lmh::ImgArgs A)
{
    __shared__ TileSmem sm;
    const int u = A.u;
    const PassMode m = pass_mode(A, u);
    if ((m.prior && A.skip_prior) || (m.data && !m.init && A.skip_data)) return;  // the other pass serves it
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) reset_next_slot(A, u);
    for (int64_t t = blockIdx.x; t < n_tiles(A.n[0], A.n[1], A.n[2]); t += gridDim.x)
        image_tile(A, m, u, tile_of(t, A.n[0], A.n[1]), A.x_cur, A.x_nxt_std, A.x_nxt_yf, sm);
}

// Image passes of every active frame of a batch at update u: work items are
// (frame, tile) pairs; x alternates between the frame's two buffers.
__global__ void __launch_bounds__(256) image_batch_kernel(const lmh::BatchImgArgs B)
{
    __shared__ TileSmem sm;
    const int par = B.u & 1;
    for (int64_t t = blockIdx.x; t < (int64_t)B.cap * B.tiles_per_slot; t += gridDim.x) {
        const int s = (int)(t / B.tiles_per_slot);
        if (!B.active[s]) continue;
        const lmh::ImgArgs& A = B.slots[s];
        const int64_t lt = t - (int64_t)s * B.tiles_per_slot;
        const PassMode m = pass_mode(A, B.u);
        if (lt == 0 && threadIdx.x == 0 && threadIdx.y == 0) reset_next_slot(A, B.u);
        image_tile(A, m, B.u, tile_of(lt, A.n[0], A.n[1]), A.xbuf[par], A.xbuf[par ^ 1], A.xbuf_yf[par ^ 1], sm);
    }
}

// ---- TMA-staged image passes ---------------------------------------------
// A block owns a 32 x 32 column of the x-y plane and a run of z slices and
// marches through them.  While slice z is computed, the tensor memory
// accelerator fetches the inputs of slice z+1 into the other half of a
// two-stage shared-memory ring (one thread issues the copies, an mbarrier
// counts their bytes), so each block keeps a whole slice of loads in flight
// without holding them in registers.  Data updates merge the accumulators
// into z; prior updates fuse the prior's dual step (Alg. 2: w+ from
// x over the tile and a one-voxel halo), dz = K^T(w+ - w) and the primal
// step into the same pass, and the event kernel does nothing for them.
// Needs rows of a multiple of 4 floats (16-byte tensor strides) and
// nx >= 40, ny >= 36 (boxes inside the tensor); other grids use
// image_pass_kernel.  Results equal image_pass_kernel's (and the event
// kernel's prior step) bit for bit: same operations in the same order.

constexpr int XHW = 40, XHH = 34;  // x halo box: x0-4 .. x0+35, y0-1 .. y0+32
constexpr int WBW = 36, WBH = 33;  // w box: x0-4 .. x0+31, y0-1 .. y0+31 (per component)
constexpr int EW = 33;             // region of w+: x0-1 .. x0+31, y0-1 .. y0+31
constexpr int EWW = EW * EW;
constexpr int TP = 33;             // pitch of the transposed tiles

struct TmaLayout {  // byte offsets into dynamic shared memory
    static constexpr int bars = 0;
    static constexpr int xh = 128;  // ring of 3 x-halo slices
    static constexpr int xh_sz = 5504;
    static constexpr int stage = xh + 3 * xh_sz;  // 2 stages
    static constexpr int stage_sz = 32768;
    // prior stage: w (<= 3 components), T, z, zc
    static constexpr int p_wc = 0, p_T = 14336, p_z = p_T + 4096, p_zc = p_z + 4096;
    // data stage: acc_std, acc_yf (u64 when deterministic), x, T, z, zc
    static constexpr int d_as = 0, d_ay = 8192, d_x = 16384, d_T = 20480, d_z = 24576, d_zc = 28672;
    static constexpr int dbuf = stage + 2 * stage_sz;  // w+ - w (3 x 33 x 33 floats) / transposed acc_yf
    static constexpr int dbuf_sz = 13184;
    static constexpr int xo = dbuf + dbuf_sz;  // transposed x tile
    static constexpr int xo_sz = 4224;
    static constexpr int total = xo + xo_sz;
};
static_assert(TmaLayout::p_zc + 4096 <= TmaLayout::stage_sz, "prior stage");
static_assert(TmaLayout::d_zc + 4096 <= TmaLayout::stage_sz, "data stage");
static_assert(XHW * XHH * 4 <= TmaLayout::xh_sz && 3 * EWW * 4 <= TmaLayout::dbuf_sz &&
                  TD * TP * 8 <= TmaLayout::dbuf_sz && TD * TP * 4 <= TmaLayout::xo_sz,
              "buffers");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Orders this thread's earlier shared-memory accesses before later
// asynchronous-proxy (TMA) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// The maps live in global memory and are rewritten by the host when a state
// is created (possibly at the address of a destroyed state's maps): make the
// tensor-map proxy read the current contents before a copy uses them.
__device__ __forceinline__ void tmap_acquire(const CUtensorMap* m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

// Two-stage ring state: stage parities and the block's abort flag.
struct Pipe {
    uint64_t* bar;
    uint32_t ph;
    int* abort;
};

// Bounded wait for stage s; a wait that gives up marks the block aborted
// and sets *err.  Ends with a block barrier, so the result is uniform.
__device__ __forceinline__ bool stage_wait(Pipe& p, int s, unsigned* err)
{
    const uint32_t par = (p.ph >> s) & 1u;
    bool ok = false;
    for (int i = 0; i < (1 << 22) && !ok; ++i) ok = mbar_try_wait(p.bar + s, par);
    p.ph ^= 1u << s;
    if (!ok) {
        *p.abort = 1;
        if (err) atomicOr(err, 1u);
    }
    __syncthreads();
    return *p.abort == 0;
}

struct Item {
    int x0, y0, zb, ze;
};

__device__ __forceinline__ int64_t tma_items(const lmh::ImgArgs& A)
{
    const int ncol = ((A.n[0] + TD - 1) / TD) * ((A.n[1] + TD - 1) / TD);
    return (int64_t)ncol * ((A.n[2] + A.zlen - 1) / A.zlen);
}

__device__ __forceinline__ Item item_of(const lmh::ImgArgs& A, int64_t it)
{
    const int ncx = (A.n[0] + TD - 1) / TD, ncol = ncx * ((A.n[1] + TD - 1) / TD);
    const int col = (int)(it % ncol), ch = (int)(it / ncol);
    Item r;
    r.x0 = (col % ncx) * TD;
    r.y0 = (col / ncx) * TD;
    r.zb = ch * A.zlen;
    r.ze = min(A.n[2], r.zb + A.zlen);
    return r;
}

// Copies of one slice (thread 0).  Prior: x slices z (first only) and z+1
// with halo, w(z) with halo and, for slices the block owns, T, z, zc (the
// directional TV's field is read with plain loads where it is needed).
// Data: both accumulators, x, T, z, zc of the tile.
__device__ __forceinline__ void issue_slice(const lmh::ImgArgs& A, bool prior, int xcur, int wp, uint8_t* sm, int s,
                                            int z, int zs, const Item& I, bool first, uint64_t* bar)
{
    const lmh::TmaMaps* M = A.tm;
    uint8_t* st = sm + TmaLayout::stage + s * TmaLayout::stage_sz;
    const uint32_t tile = TD * TD * 4;
    if (first) {
        if (prior) {
            tmap_acquire(&M->xh[xcur]);
            tmap_acquire(&M->w[wp]);
        } else {
            tmap_acquire(&M->acc_std);
            tmap_acquire(&M->acc_yf);
            tmap_acquire(&M->xt[xcur]);
        }
        tmap_acquire(&M->T);
        tmap_acquire(&M->z);
        tmap_acquire(&M->zc);
    }
    fence_proxy_async();
    if (prior) {
        const bool own = z >= I.zb;
        const uint32_t xb = XHW * XHH * 4, wb = (uint32_t)(WBW * WBH * A.ndim * 4);
        const uint32_t bytes = xb * (first ? 2u : 1u) + wb + (own ? tile * (A.kahan ? 3u : 2u) : 0u);
        mbar_expect_tx(bar + s, bytes);
        const CUtensorMap* xm = &M->xh[xcur];
        if (first) tma_load_3d(sm + TmaLayout::xh + ((z - zs) % 3) * TmaLayout::xh_sz, xm, I.x0 - 4, I.y0 - 1, z, bar + s);
        tma_load_3d(sm + TmaLayout::xh + ((z + 1 - zs) % 3) * TmaLayout::xh_sz, xm, I.x0 - 4, I.y0 - 1, z + 1,
                    bar + s);
        tma_load_4d(st + TmaLayout::p_wc, &M->w[wp], I.x0 - 4, I.y0 - 1, z, 0, bar + s);
        if (own) {
            tma_load_3d(st + TmaLayout::p_T, &M->T, I.x0, I.y0, z, bar + s);
            tma_load_3d(st + TmaLayout::p_z, &M->z, I.x0, I.y0, z, bar + s);
            if (A.kahan) tma_load_3d(st + TmaLayout::p_zc, &M->zc, I.x0, I.y0, z, bar + s);
        }
    } else {
        // accumulator tiles: u64 (deterministic) or float z pairs, 8 KB each
        const uint32_t acc = (A.det || A.acc_pairs) ? 2 * tile : tile;
        const int ax = A.acc_pairs && !A.det ? 2 : 1;  // pair tensors are (2n, ., .)
        if (z < I.zb) {
            // halo slice below the run: only the upper halves of its accumulator pairs are needed
            mbar_expect_tx(bar + s, 2 * acc);
            tma_load_3d(st + TmaLayout::d_as, &M->acc_std, ax * I.x0, I.y0, z, bar + s);
            tma_load_3d(st + TmaLayout::d_ay, &M->acc_yf, ax * I.y0, I.x0, z, bar + s);
            return;
        }
        mbar_expect_tx(bar + s, 2 * acc + 3 * tile + (A.kahan ? tile : 0u));
        tma_load_3d(st + TmaLayout::d_as, &M->acc_std, ax * I.x0, I.y0, z, bar + s);
        tma_load_3d(st + TmaLayout::d_ay, &M->acc_yf, ax * I.y0, I.x0, z, bar + s);
        tma_load_3d(st + TmaLayout::d_x, &M->xt[xcur], I.x0, I.y0, z, bar + s);
        tma_load_3d(st + TmaLayout::d_T, &M->T, I.x0, I.y0, z, bar + s);
        tma_load_3d(st + TmaLayout::d_z, &M->z, I.x0, I.y0, z, bar + s);
        if (A.kahan) tma_load_3d(st + TmaLayout::d_zc, &M->zc, I.x0, I.y0, z, bar + s);
    }
}

// z update, zbar and the primal step at one voxel (same operations as
// image_tile).
__device__ __forceinline__ float primal_step(float x0, float tm, float z0, float zl0, float dz, float inv_p, bool kahan,
                                             float& zh, float& zl)
{
    zl = 0.0f;
    if (kahan) {
        float e;
        two_sum(z0, dz, zh, e);
        zl = zl0 + e;
    } else {
        zh = z0 + dz;
    }
    const float zbar = fmaf(dz, inv_p, zh + zl);
    return fmaxf(0.0f, fmaf(-tm, zbar, x0));
}

// Writes the transposed x tile of slice z to the y-fastest copy.
__device__ __forceinline__ void store_x_yf(const lmh::ImgArgs& A, const float* XO, float* x_nxt_yf, const Item& I,
                                           int z)
{
    const int nx = A.n[0], ny = A.n[1];
    const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = wrow + 8 * k;  // x offset
        const int ix = I.x0 + r, iy = I.y0 + lane;
        if (ix < nx && iy < ny) x_nxt_yf[((int64_t)z * nx + ix) * ny + iy] = XO[lane * TP + r];
    }
}

// Fused prior update for slice z of item I (z < I.zb: halo slice, only the
// z component of w+ - w is kept for the next slice).
__device__ __forceinline__ void prior_slice(const lmh::ImgArgs& A, int wp, uint8_t* sm, int s, int z, int zs,
                                            const Item& I, float* dprev, float* x_nxt_std, float* x_nxt_yf)
{
    const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
    const int64_t V = A.V;
    const bool hz = nz > 1;
    const bool own = z >= I.zb;
    const float* X0 = (const float*)(sm + TmaLayout::xh + ((z - zs) % 3) * TmaLayout::xh_sz);
    const float* X1 = (const float*)(sm + TmaLayout::xh + ((z + 1 - zs) % 3) * TmaLayout::xh_sz);
    const uint8_t* st = sm + TmaLayout::stage + s * TmaLayout::stage_sz;
    const float* WC = (const float*)(st + TmaLayout::p_wc);
    float* D = (float*)(sm + TmaLayout::dbuf);
    float* XO = (float*)(sm + TmaLayout::xo);
    float* wn = A.w_nxt[wp];
    const float sp = A.s_prior, beta = A.beta;
    const float* xi = A.xi;  // directional TV: the structural field [3][V] (3D grids), else nullptr
    // w+ = v / max(1, |v|/beta), v = w + S K x, over the tile (4 points per
    // thread) and its -1 halo (row y0-1 and column x0-1: 65 points), and
    // D = K^T's operand w+ - w; the directional TV takes the part of the
    // difference vector perpendicular to the field before v and again of
    // w+ - w (D = P (w+ - w)), in the order of the event kernel's dual step
    // the field at the thread's points (4 of the tile, at most one of the
    // halo), all loads issued before any arithmetic
    const int lane0 = threadIdx.x & 31, wrow0 = threadIdx.x >> 5, t0 = threadIdx.x;
    float fxr[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, fyr[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
          fzr[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (xi != nullptr) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            int ex, ey;
            if (k < 4) {
                ex = lane0 + 1;
                ey = wrow0 + 8 * k + 1;
            } else {
                ex = t0 < EW ? t0 : 0;
                ey = t0 < EW ? 0 : t0 - EW + 1;
            }
            const int ix = I.x0 - 1 + ex, iy = I.y0 - 1 + ey;
            if ((k < 4 || t0 < 2 * EW - 1) && ix >= 0 && iy >= 0 && ix < nx && iy < ny) {
                const int64_t j = ((int64_t)z * ny + iy) * nx + ix;
                fxr[k] = __ldg(xi + j);
                fyr[k] = __ldg(xi + V + j);
                if (hz) fzr[k] = __ldg(xi + 2 * V + j);
            }
        }
    }
    auto wplus = [&](int ex, int ey, bool tile_pt, int k) {
        const int ix = I.x0 - 1 + ex, iy = I.y0 - 1 + ey;
        float dx = 0.0f, dy = 0.0f, dzc = 0.0f;
        if (ix >= 0 && iy >= 0 && ix < nx && iy < ny) {
            const int xb = ey * XHW + ex + 3;
            const int wb = ey * WBW + ex + 3;
            const float xc = X0[xb];
            const float wx = WC[wb], wy = WC[WBW * WBH + wb];
            float gx = ix < nx - 1 ? X0[xb + 1] - xc : 0.0f;
            float gy = iy < ny - 1 ? X0[xb + XHW] - xc : 0.0f;
            float gz = hz ? (z < nz - 1 ? X1[xb] - xc : 0.0f) : 0.0f;
            const float fx = fxr[k], fy = fyr[k], fz = fzr[k];
            if (xi != nullptr) dtv_perp(fx, fy, fz, gx, gy, gz);
            const float vx = fmaf(sp, gx, wx);
            const float vy = fmaf(sp, gy, wy);
            float vz = 0.0f, wz = 0.0f;
            if (hz) {
                wz = WC[2 * WBW * WBH + wb];
                vz = fmaf(sp, gz, wz);
            }
            const float sc = tv_ball_scale(fmaf(vx, vx, fmaf(vy, vy, vz * vz)), beta);
            // rounded products (never fused into the differences below), as stored by the plain path
            const float ox = __fmul_rn(vx, sc), oy = __fmul_rn(vy, sc), oz = __fmul_rn(vz, sc);
            dx = ox - wx;
            dy = oy - wy;
            dzc = hz ? oz - wz : 0.0f;
            if (xi != nullptr) dtv_perp(fx, fy, fz, dx, dy, dzc);
            if (own && tile_pt) {
                const int64_t j = ((int64_t)z * ny + iy) * nx + ix;
                wn[j] = ox;
                wn[V + j] = oy;
                if (hz) wn[2 * V + j] = oz;
            }
        }
        const int p = ey * EW + ex;
        D[p] = dx;
        D[EWW + p] = dy;
        D[2 * EWW + p] = dzc;
    };
    {
        const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 4; ++k) wplus(lane + 1, wrow + 8 * k + 1, true, k);
        const int t = threadIdx.x;
        if (t < EW) wplus(t, 0, false, 4);
        else if (t < 2 * EW - 1) wplus(0, t - EW + 1, false, 4);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
    const float* Tt = (const float*)(st + TmaLayout::p_T);
    const float* Zt = (const float*)(st + TmaLayout::p_z);
    const float* ZCt = (const float*)(st + TmaLayout::p_zc);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ty = wrow + 8 * k, tx = lane;
        const int ix = I.x0 + tx, iy = I.y0 + ty;
        const int e = (ty + 1) * EW + tx + 1;
        if (own && ix < nx && iy < ny) {
            // dz = (K^T (w+ - w))_j, component order and signs of prior_dz
            float dz = 0.0f;
            if (ix < nx - 1) dz -= D[e];
            if (ix >= 1) dz += D[e - 1];
            if (iy < ny - 1) dz -= D[EWW + e];
            if (iy >= 1) dz += D[EWW + e - EW];
            if (hz) {
                if (z < nz - 1) dz -= D[2 * EWW + e];
                if (z >= 1) dz += dprev[k];
            }
            const int t = ty * TD + tx;
            float zh, zl;
            const float xn = primal_step(X0[(ty + 1) * XHW + tx + 4], Tt[t], Zt[t], A.kahan ? ZCt[t] : 0.0f, dz,
                                         A.inv_p_prior, A.kahan != 0, zh, zl);
            const int64_t j = ((int64_t)z * ny + iy) * nx + ix;
            A.z[j] = zh;
            if (A.kahan) A.zc[j] = zl;
            x_nxt_std[j] = xn;
            XO[ty * TP + tx] = xn;
        }
        dprev[k] = hz ? D[2 * EWW + e] : 0.0f;
    }
    if (own) {
        __syncthreads();
        store_x_yf(A, XO, x_nxt_yf, I, z);
    }
}

// Data update merge for slice z of item I.  Float accumulators are z pairs:
// a voxel's value is the first half of its own pair plus the second half of
// the pair below, which the thread carries from the previous slice in
// prev_s (its 4 x-fastest points) and prev_y (its 4 y-fastest points).  A run
// starting above z = 0 first reads the slice below (z < I.zb) for these only.
__device__ __forceinline__ void data_slice(const lmh::ImgArgs& A, const PassMode& m, uint8_t* sm, int s, int z,
                                           const Item& I, float* x_nxt_std, float* x_nxt_yf, float* prev_s,
                                           float* prev_y)
{
    const int nx = A.n[0], ny = A.n[1];
    const int64_t sz = (int64_t)nx * ny;
    const bool det = A.det != 0;
    const bool pairs = A.acc_pairs && !det;
    const uint8_t* st = sm + TmaLayout::stage + s * TmaLayout::stage_sz;
    const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
    float* AYT = (float*)(sm + TmaLayout::dbuf);
    long long* AYT64 = (long long*)(sm + TmaLayout::dbuf);
    float* XO = (float*)(sm + TmaLayout::xo);
    const float* AYp = (const float*)(st + TmaLayout::d_ay);
    const float* ASp = (const float*)(st + TmaLayout::d_as);
    if (z < I.zb) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = wrow + 8 * k;
            prev_y[k] = AYp[r * 2 * TD + 2 * lane + 1];
            prev_s[k] = ASp[r * 2 * TD + 2 * lane + 1];
        }
        return;
    }
    const bool below = z > 0;
    // acc_yf tile (rows x, columns y) -> transposed buffer [y][x]; clear it in memory
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = wrow + 8 * k, c = lane;
        const int ix = I.x0 + r, iy = I.y0 + c;
        if (det) {
            AYT64[c * TP + r] = ((const long long*)(st + TmaLayout::d_ay))[r * TD + c];
        } else if (pairs) {
            AYT[c * TP + r] = AYp[r * 2 * TD + 2 * c] + prev_y[k];
            prev_y[k] = AYp[r * 2 * TD + 2 * c + 1];
        } else {
            AYT[c * TP + r] = AYp[r * TD + c];
        }
        if (ix < nx && iy < ny) {
            const int64_t k2 = ((int64_t)z * nx + ix) * ny + iy;
            if (det) {
                A.acci_yf[k2] = 0ULL;
            } else if (pairs) {
                A.acc_yf[2 * k2] = 0.0f;
                if (below) A.acc_yf[2 * (k2 - sz) + 1] = 0.0f;
            } else {
                A.acc_yf[k2] = 0.0f;
            }
        }
    }
    __syncthreads();
    const float* Xt = (const float*)(st + TmaLayout::d_x);
    const float* Tt = (const float*)(st + TmaLayout::d_T);
    const float* Zt = (const float*)(st + TmaLayout::d_z);
    const float* ZCt = (const float*)(st + TmaLayout::d_zc);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ty = wrow + 8 * k, tx = lane;
        const int ix = I.x0 + tx, iy = I.y0 + ty;
        if (ix < nx && iy < ny) {
            const int t = ty * TD + tx;
            const int64_t j = ((int64_t)z * ny + iy) * nx + ix;
            float dz;
            if (det) {
                long long sacc = ((const long long*)(st + TmaLayout::d_as))[t];
                sacc += AYT64[ty * TP + tx];
                dz = (float)((double)sacc * m.fx);
                A.acci_std[j] = 0ULL;
            } else if (pairs) {
                dz = ASp[ty * 2 * TD + 2 * tx] + prev_s[k];
                dz += AYT[ty * TP + tx];
                A.acc_std[2 * j] = 0.0f;
                if (below) A.acc_std[2 * (j - sz) + 1] = 0.0f;
            } else {
                dz = ASp[t];
                dz += AYT[ty * TP + tx];
                A.acc_std[j] = 0.0f;
            }
            float zh, zl;
            const float xn =
                primal_step(Xt[t], Tt[t], Zt[t], A.kahan ? ZCt[t] : 0.0f, dz, m.inv_p, A.kahan != 0, zh, zl);
            A.z[j] = zh;
            if (A.kahan) A.zc[j] = zl;
            x_nxt_std[j] = xn;
            XO[ty * TP + tx] = xn;
        }
        if (pairs) prev_s[k] = ASp[ty * 2 * TD + 2 * tx + 1];
    }
    __syncthreads();
    store_x_yf(A, XO, x_nxt_yf, I, z);
}

// One work item: its slices in order, inputs of slice z+1 in flight while
// slice z is computed.  Returns false if a wait gave up.
__device__ bool tma_item(const lmh::ImgArgs& A, const PassMode& m, int u, int64_t it, int xcur, float* x_nxt_std,
                         float* x_nxt_yf, uint8_t* sm, Pipe& p)
{
    const Item I = item_of(A, it);
    const bool prior = m.prior;
    const int wp = prior ? A.wpar[u] : 0;
    // a halo slice below the run: the prior needs its w+, paired accumulators their upper halves
    const bool halo = I.zb > 0 && (prior || (A.acc_pairs && !A.det));
    const int zs = halo ? I.zb - 1 : I.zb;
    float dprev[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float prev_y[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (threadIdx.x == 0) issue_slice(A, prior, xcur, wp, sm, 0, zs, zs, I, true, p.bar);
    for (int z = zs, i = 0; z < I.ze; ++z, ++i) {
        const int s = i & 1;
        if (threadIdx.x == 0 && z + 1 < I.ze) issue_slice(A, prior, xcur, wp, sm, s ^ 1, z + 1, zs, I, false, p.bar);
        if (!stage_wait(p, s, A.err)) return false;
        if (prior) prior_slice(A, wp, sm, s, z, zs, I, dprev, x_nxt_std, x_nxt_yf);
        else data_slice(A, m, sm, s, z, I, x_nxt_std, x_nxt_yf, dprev, prev_y);
        __syncthreads();
    }
    return true;
}

__device__ __forceinline__ void tma_block_init(uint8_t* sm, int* abort_flag)
{
    if (threadIdx.x == 0) {
        uint64_t* bar = (uint64_t*)(sm + TmaLayout::bars);
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256, 2) image_tma_kernel(const lmh::ImgArgs A)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ int abort_flag;
    tma_block_init(sm, &abort_flag);
    Pipe p{(uint64_t*)(sm + TmaLayout::bars), 0u, &abort_flag};
    const int u = A.u;
    const PassMode m = pass_mode(A, u);
    if ((m.prior && A.skip_prior) || (m.data && !m.init && A.skip_data)) return;  // the other pass serves it
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_next_slot(A, u);
    const int64_t n = tma_items(A);
    for (int64_t it = blockIdx.x; it < n; it += gridDim.x)
        if (!tma_item(A, m, u, it, A.xcur, A.x_nxt_std, A.x_nxt_yf, sm, p)) break;
}

// Batched epochs: work items (frame, column, z run) over the active frames.
__global__ void __launch_bounds__(256, 2) image_tma_batch_kernel(const lmh::BatchImgArgs B)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ int abort_flag;
    tma_block_init(sm, &abort_flag);
    Pipe p{(uint64_t*)(sm + TmaLayout::bars), 0u, &abort_flag};
    // the frame's arguments in shared memory: the item code reads them in its inner loops
    __shared__ lmh::ImgArgs sA;
    int cur = -1;
    const int par = B.u & 1;
    for (int64_t t = blockIdx.x; t < (int64_t)B.cap * B.tiles_per_slot; t += gridDim.x) {
        const int s = (int)(t / B.tiles_per_slot);
        if (!B.active[s]) continue;
        if (s != cur) {
            __syncthreads();  // no thread still reads the previous frame's arguments
            if (threadIdx.x == 0) sA = B.slots[s];
            __syncthreads();
            cur = s;
        }
        const lmh::ImgArgs& A = sA;
        const int64_t lt = t - (int64_t)s * B.tiles_per_slot;
        const PassMode m = pass_mode(A, B.u);
        if (lt == 0 && threadIdx.x == 0) reset_next_slot(A, B.u);
        if (!tma_item(A, m, B.u, lt, par, A.xbuf[par ^ 1], A.xbuf_yf[par ^ 1], sm, p)) break;
    }
}

// Prefix parity of the w buffers for every active frame of a batch.
__global__ void wpar_batch_kernel(const lmh::BatchImgArgs B, int count)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B.cap || !B.active[s]) return;
    const lmh::ImgArgs& A = B.slots[s];
    int p = *A.wbase;
    int* wpar = A.wpar_w;
    wpar[0] = p;
    for (int u = 0; u < count; ++u) {
        if (A.seq[u] >= A.n_subsets) p ^= 1;
        wpar[u + 1] = p;
    }
    *A.wbase = p;
}

int tile_grid(const lm_grid* g, int per_sm = 8)
{
    const int64_t nt = (int64_t)((g->n[0] + TD - 1) / TD) * ((g->n[1] + TD - 1) / TD) * g->n[2];
    return (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)lmh::num_sms() * per_sm));
}

__global__ void wpar_kernel(const uint16_t* seq, int count, int n_subsets, int* wpar, int* wbase)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int p = *wbase;
        wpar[0] = p;
        for (int u = 0; u < count; ++u) {
            if (seq[u] >= n_subsets) p ^= 1;
            wpar[u + 1] = p;
        }
        *wbase = p;
    }
}

__global__ void step_T_kernel(const float* __restrict__ sens, float* __restrict__ T, int64_t V, float t_prior,
                              float c_data)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const float s = sens[j];
        const float t_data = s > 0.0f ? c_data / s : INFINITY;
        T[j] = fminf(t_data, t_prior);
    }
}

constexpr int RB = 1024;  // blocks of the fixed-shape reductions

// partial min / max (fixed grid of RB blocks; deterministic)
__global__ void __launch_bounds__(256) minmax_partial(const float* __restrict__ x, int64_t n, float* part)
{
    __shared__ float smn[256], smx[256];
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)RB * 256) {
        const float v = x[i];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smn[threadIdx.x] = fminf(smn[threadIdx.x], smn[threadIdx.x + s]);
            smx[threadIdx.x] = fmaxf(smx[threadIdx.x], smx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = smn[0];
        part[RB + blockIdx.x] = smx[0];
    }
}

__global__ void __launch_bounds__(256) minmax_final(float* part)
{
    __shared__ float smn[256], smx[256];
    float mn = INFINITY, mx = -INFINITY;
    for (int i = threadIdx.x; i < RB; i += 256) {
        mn = fminf(mn, part[i]);
        mx = fmaxf(mx, part[RB + i]);
    }
    smn[threadIdx.x] = mn;
    smx[threadIdx.x] = mx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smn[threadIdx.x] = fminf(smn[threadIdx.x], smn[threadIdx.x + s]);
            smx[threadIdx.x] = fmaxf(smx[threadIdx.x], smx[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * RB] = smn[0];
        part[2 * RB + 1] = smx[0];
    }
}

__device__ __forceinline__ double block_sum_d(double v, double* sm)
{
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sm[0];
    __syncthreads();
    return r;
}

// objective parts over voxels: <sens, x> and ||Kx||_{2,1} (FP64); K is the
// forward difference, or its part perpendicular to the field xi (DTV)
__global__ void __launch_bounds__(256) obj_img_partial(const float* __restrict__ sens, const float* __restrict__ x,
                                                       const float* __restrict__ xi, int nx, int ny, int nz,
                                                       double* part)
{
    __shared__ double sm[256];
    const int64_t V = (int64_t)nx * ny * nz;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x; j < V; j += (int64_t)RB * 256) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        const double xj = (double)x[j];
        s1 += (double)sens[j] * xj;
        double gx = 0.0, gy = 0.0, gz = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        int c = 0;
        if (nx > 1) {
            if (ix < nx - 1) gx = (double)x[j + 1] - xj;
            if (xi) fx = xi[c * V + j];
            ++c;
        }
        if (ny > 1) {
            if (iy < ny - 1) gy = (double)x[j + nx] - xj;
            if (xi) fy = xi[c * V + j];
            ++c;
        }
        if (nz > 1) {
            if (iz < nz - 1) gz = (double)x[j + (int64_t)nx * ny] - xj;
            if (xi) fz = xi[c * V + j];
        }
        if (xi) {
            const double t = fx * gx + fy * gy + fz * gz;
            gx -= fx * t;
            gy -= fy * t;
            gz -= fz * t;
        }
        s2 += sqrt(gx * gx + gy * gy + gz * gz);
    }
    s1 = block_sum_d(s1, sm);
    s2 = block_sum_d(s2, sm);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = s1;
        part[RB + blockIdx.x] = s2;
    }
}

// sum_e w_e log(p_e + s_e) and, with weights (sinogram bins: w = d_b), sum_e s_e (FP64)
__global__ void __launch_bounds__(256) obj_ev_partial(const float* __restrict__ p, const float* __restrict__ s,
                                                      float s_flat, const uint16_t* __restrict__ w, int64_t n,
                                                      double* part)
{
    __shared__ double sm[256];
    double acc = 0.0, acs = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)RB * 256) {
        const double se = s ? (double)s[e] : (double)s_flat;
        if (w) {
            if (w[e]) acc += (double)w[e] * log((double)p[e] + se);
            acs += se;
        } else {
            acc += log((double)p[e] + se);
        }
    }
    acc = block_sum_d(acc, sm);
    acs = block_sum_d(acs, sm);
    if (threadIdx.x == 0) {
        part[2 * RB + blockIdx.x] = acc;
        part[3 * RB + blockIdx.x] = acs;
    }
}

__global__ void __launch_bounds__(256) obj_final(double* part)
{
    __shared__ double sm[256];
    for (int q = 0; q < 4; ++q) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < RB; i += 256) acc += part[q * RB + i];
        acc = block_sum_d(acc, sm);
        if (threadIdx.x == 0) part[4 * RB + q] = acc;
    }
}

// ---- directional TV (standalone calls) ----
// Difference vector of x at voxel j (0 for boundary differences), axis order.
__device__ __forceinline__ void fwd_diff(const float* x, int64_t j, int ix, int iy, int iz, int nx, int ny, int nz,
                                         float& gx, float& gy, float& gz)
{
    const float xj = x[j];
    gx = (nx > 1 && ix < nx - 1) ? x[j + 1] - xj : 0.0f;
    gy = (ny > 1 && iy < ny - 1) ? x[j + nx] - xj : 0.0f;
    gz = (nz > 1 && iz < nz - 1) ? x[j + (int64_t)nx * ny] - xj : 0.0f;
}

// Field components of voxel j per axis (0 for axes of length 1).
__device__ __forceinline__ void field_at(const float* xi, int64_t V, int64_t j, int nx, int ny, int nz, float& fx,
                                         float& fy, float& fz)
{
    int c = 0;
    fx = nx > 1 ? xi[(c++) * V + j] : 0.0f;
    fy = ny > 1 ? xi[(c++) * V + j] : 0.0f;
    fz = nz > 1 ? xi[(c++) * V + j] : 0.0f;
}

__device__ __forceinline__ void store_comps(float* g, int64_t V, int64_t j, int nx, int ny, int nz, float gx, float gy,
                                            float gz)
{
    int c = 0;
    if (nx > 1) g[(c++) * V + j] = gx;
    if (ny > 1) g[(c++) * V + j] = gy;
    if (nz > 1) g[(c++) * V + j] = gz;
}

// xi_j = (grad v)_j / sqrt(|(grad v)_j|^2 + eta^2), 0 where both vanish
__global__ void dtv_field_kernel(const float* __restrict__ v, float eta2, float* __restrict__ xi, int nx, int ny,
                                 int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        float gx, gy, gz;
        fwd_diff(v, j, ix, iy, iz, nx, ny, nz, gx, gy, gz);
        const float n2 = fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, eta2)));
        const float r = n2 > 0.0f ? 1.0f / sqrtf(n2) : 0.0f;
        store_comps(xi, V, j, nx, ny, nz, gx * r, gy * r, gz * r);
    }
}

// g = K x = P grad x
__global__ void dtv_grad_kernel(const float* __restrict__ x, const float* __restrict__ xi, float* __restrict__ g,
                                int nx, int ny, int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        float gx, gy, gz, fx, fy, fz;
        fwd_diff(x, j, ix, iy, iz, nx, ny, nz, gx, gy, gz);
        field_at(xi, V, j, nx, ny, nz, fx, fy, fz);
        dtv_perp(fx, fy, fz, gx, gy, gz);
        store_comps(g, V, j, nx, ny, nz, gx, gy, gz);
    }
}

// (P g) at voxel m
__device__ __forceinline__ void pg_at(const float* g, const float* xi, int64_t V, int64_t m, int nx, int ny, int nz,
                                      float& px, float& py, float& pz)
{
    float fx, fy, fz;
    field_at(g, V, m, nx, ny, nz, px, py, pz);
    field_at(xi, V, m, nx, ny, nz, fx, fy, fz);
    dtv_perp(fx, fy, fz, px, py, pz);
}

// d = -K^T g = div (P g)
__global__ void dtv_div_kernel(const float* __restrict__ g, const float* __restrict__ xi, float* __restrict__ d,
                               int nx, int ny, int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        float px, py, pz, qx, qy, qz;
        pg_at(g, xi, V, j, nx, ny, nz, px, py, pz);
        float s = 0.0f;
        if (nx > 1) {
            if (ix < nx - 1) s += px;
            if (ix >= 1) {
                pg_at(g, xi, V, j - 1, nx, ny, nz, qx, qy, qz);
                s -= qx;
            }
        }
        if (ny > 1) {
            if (iy < ny - 1) s += py;
            if (iy >= 1) {
                pg_at(g, xi, V, j - nx, nx, ny, nz, qx, qy, qz);
                s -= qy;
            }
        }
        if (nz > 1) {
            if (iz < nz - 1) s += pz;
            if (iz >= 1) {
                pg_at(g, xi, V, j - (int64_t)nx * ny, nx, ny, nz, qx, qy, qz);
                s -= qz;
            }
        }
        d[j] = s;
    }
}

// ---- TV operators (standalone calls) ----
__global__ void tv_grad_kernel(const float* __restrict__ x, float* __restrict__ g, int nx, int ny, int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        const float xj = x[j];
        int c = 0;
        if (nx > 1) g[(c++) * V + j] = ix < nx - 1 ? x[j + 1] - xj : 0.0f;
        if (ny > 1) g[(c++) * V + j] = iy < ny - 1 ? x[j + nx] - xj : 0.0f;
        if (nz > 1) g[(c++) * V + j] = iz < nz - 1 ? x[j + (int64_t)nx * ny] - xj : 0.0f;
    }
}

// d = div g = -K^T g
__global__ void tv_div_kernel(const float* __restrict__ g, float* __restrict__ d, int nx, int ny, int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / ((int64_t)nx * ny));
        float s = 0.0f;
        int c = 0;
        if (nx > 1) {
            const float* q = g + (int64_t)(c++) * V;
            if (ix < nx - 1) s += q[j];
            if (ix >= 1) s -= q[j - 1];
        }
        if (ny > 1) {
            const float* q = g + (int64_t)(c++) * V;
            if (iy < ny - 1) s += q[j];
            if (iy >= 1) s -= q[j - nx];
        }
        if (nz > 1) {
            const float* q = g + (int64_t)(c++) * V;
            if (iz < nz - 1) s += q[j];
            if (iz >= 1) s -= q[j - (int64_t)nx * ny];
        }
        d[j] = s;
    }
}

__global__ void tv_prox_kernel(float* __restrict__ w, int64_t V, int ndim, float beta)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        float s2 = 0.0f;
        for (int c = 0; c < ndim; ++c) s2 = fmaf(w[c * V + j], w[c * V + j], s2);
        const float nrm = sqrtf(s2);
        if (beta > 0.0f) {
            const float den = fmaxf(1.0f, nrm / beta);
            for (int c = 0; c < ndim; ++c) w[c * V + j] = w[c * V + j] / den;
        } else {
            for (int c = 0; c < ndim; ++c) w[c * V + j] = 0.0f;
        }
    }
}

// ---- ||K|| power iteration (FP64) ----
__global__ void kn_init(double* v, int nx, int ny, int nz)
{
    const int64_t V = (int64_t)nx * ny * nz;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(j % nx) + (int)((j / nx) % ny) + (int)(j / ((int64_t)nx * ny));
        v[j] = (s & 1) ? -1.0 : 1.0;
    }
}

// u = K^T K (c v), c = scal[0]; partial sums of (cv).u, (cv).(cv), u.u
__global__ void __launch_bounds__(256) kn_apply(const double* __restrict__ v, double* __restrict__ u,
                                                const double* __restrict__ scal, int nx, int ny, int nz, double* part)
{
    __shared__ double sm[256];
    const int64_t V = (int64_t)nx * ny * nz;
    const double c = scal[0];
    const int64_t sz = (int64_t)nx * ny;
    double a = 0.0, b = 0.0, q = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x; j < V; j += (int64_t)RB * 256) {
        const int ix = (int)(j % nx), iy = (int)((j / nx) % ny), iz = (int)(j / sz);
        const double vj = c * v[j];
        double r = 0.0;
        if (nx > 1) {
            if (ix >= 1) r += vj - c * v[j - 1];
            if (ix < nx - 1) r -= c * v[j + 1] - vj;
        }
        if (ny > 1) {
            if (iy >= 1) r += vj - c * v[j - nx];
            if (iy < ny - 1) r -= c * v[j + nx] - vj;
        }
        if (nz > 1) {
            if (iz >= 1) r += vj - c * v[j - sz];
            if (iz < nz - 1) r -= c * v[j + sz] - vj;
        }
        u[j] = r;
        a += vj * r;
        b += vj * vj;
        q += r * r;
    }
    a = block_sum_d(a, sm);
    b = block_sum_d(b, sm);
    q = block_sum_d(q, sm);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = a;
        part[RB + blockIdx.x] = b;
        part[2 * RB + blockIdx.x] = q;
    }
}

// scal[0] = 1/||u||, scal[1] = lambda = (v.u)/(v.v)
__global__ void __launch_bounds__(256) kn_final(const double* part, double* scal)
{
    __shared__ double sm[256];
    double r[3];
    for (int q = 0; q < 3; ++q) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < RB; i += 256) acc += part[q * RB + i];
        r[q] = block_sum_d(acc, sm);
    }
    if (threadIdx.x == 0) {
        scal[1] = r[1] > 0.0 ? r[0] / r[1] : 0.0;
        scal[0] = r[2] > 0.0 ? 1.0 / sqrt(r[2]) : 0.0;
    }
}

__global__ void zadd_kernel(const float* z, const float* zc, float* out, int64_t V)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x)
        out[j] = zc ? z[j] + zc[j] : z[j];
}

int flat_grid(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)lmh::num_sms() * 16));
}

}  // namespace

namespace lmh {

void launch_transpose_to_yf(const lm_grid* g, const float* src, float* dst, cudaStream_t st)
{
    transpose_to_yf_kernel<<<tile_grid(g), dim3(TD, TR), 0, st>>>(src, dst, g->n[0], g->n[1], g->n[2]);
    count_launch();
}

void launch_add_yf_to_std(const lm_grid* g, float* img, float* yf_acc, cudaStream_t st)
{
    add_yf_kernel<<<tile_grid(g), dim3(TD, TR), 0, st>>>(img, yf_acc, g->n[0], g->n[1], g->n[2]);
    count_launch();
}

void launch_fold_fixed(const lm_grid* g, float* img, unsigned long long* a_std, unsigned long long* a_yf,
                       const unsigned* maxbits, long long count, float stepmax, cudaStream_t st)
{
    fold_fixed_kernel<<<tile_grid(g), dim3(TD, TR), 0, st>>>(img, a_std, a_yf, maxbits, count, stepmax, g->n[0],
                                                             g->n[1], g->n[2]);
    count_launch();
}

void launch_image_pass(const ImgArgs& a, cudaStream_t st)
{
    lm_grid g;
    std::memset(&g, 0, sizeof(g));
    for (int d = 0; d < 3; ++d) g.n[d] = a.n[d];
    image_pass_kernel<<<tile_grid(&g), dim3(TD, TR), 0, st>>>(a);
    count_launch();
}

bool tma_capable(const lm_grid* g)
{
    return g->n[0] % 4 == 0 && g->n[1] % 4 == 0 && g->n[0] >= 40 && g->n[1] >= 36;
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

static void tma_attributes()
{
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(image_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaLayout::total);
        cudaFuncSetAttribute(image_tma_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TmaLayout::total);
    });
}

// rank <= 4; dims innermost first; strides in bytes for dims 1..rank-1
static int encode_one(CUtensorMap* m, CUtensorMapDataType t, int rank, void* base, const cuuint64_t* dims,
               const cuuint64_t* strides, const cuuint32_t* box)
{
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = encoder()(m, t, (cuuint32_t)rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    LM_CHECK(r == CUDA_SUCCESS, LM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LM_OK;
}

int encode_tma_maps(const lm_grid* g, float* const x[2], float* const w[2], int ndim, float* T, float* z, float* zc,
                    void* acc_std, void* acc_yf, bool det, float* dtvd, TmaMaps* out)
{
    LM_CHECK(tma_capable(g), LM_ERR_INVALID_ARG, "grid not supported by the TMA-staged image pass");
    LM_CHECK(encoder() != nullptr, LM_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    tma_attributes();
    std::memset(out, 0, sizeof(*out));
    const cuuint64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
    const cuuint64_t dims[3] = {nx, ny, nz}, strides[2] = {nx * 4, nx * ny * 4};
    const cuuint32_t box_h[3] = {XHW, XHH, 1}, box_t[3] = {TD, TD, 1};
    const CUtensorMapDataType F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    int rc;
    for (int k = 0; k < 2; ++k) {
        if ((rc = encode_one(&out->xh[k], F32, 3, x[k], dims, strides, box_h))) return rc;
        if ((rc = encode_one(&out->xt[k], F32, 3, x[k], dims, strides, box_t))) return rc;
        const cuuint64_t wd[4] = {nx, ny, nz, (cuuint64_t)ndim};
        const cuuint64_t ws[3] = {nx * 4, nx * ny * 4, nx * ny * nz * 4};
        const cuuint32_t wb[4] = {WBW, WBH, 1, (cuuint32_t)ndim};
        if ((rc = encode_one(&out->w[k], F32, 4, w[k], wd, ws, wb))) return rc;
        if (k == 0 && dtvd != nullptr && (rc = encode_one(&out->dtvd, F32, 4, dtvd, wd, ws, wb))) return rc;
    }
    if ((rc = encode_one(&out->T, F32, 3, T, dims, strides, box_t))) return rc;
    if ((rc = encode_one(&out->z, F32, 3, z, dims, strides, box_t))) return rc;
    if ((rc = encode_one(&out->zc, F32, 3, zc, dims, strides, box_t))) return rc;
    if (det) {
        // 64-bit fixed-point accumulators, one per voxel
        const CUtensorMapDataType at = CU_TENSOR_MAP_DATA_TYPE_UINT64;
        const cuuint64_t s_std[2] = {nx * 8, nx * ny * 8};
        if ((rc = encode_one(&out->acc_std, at, 3, acc_std, dims, s_std, box_t))) return rc;
        const cuuint64_t d_yf[3] = {ny, nx, nz}, s_yf[2] = {ny * 8, nx * ny * 8};
        if ((rc = encode_one(&out->acc_yf, at, 3, acc_yf, d_yf, s_yf, box_t))) return rc;
    } else {
        // float z pairs: a row of n voxels is 2n floats; a tile box covers 32 pairs
        const cuuint32_t box_p[3] = {2 * TD, TD, 1};
        const cuuint64_t d_std[3] = {2 * nx, ny, nz}, s_std[2] = {2 * nx * 4, 2 * nx * ny * 4};
        if ((rc = encode_one(&out->acc_std, F32, 3, acc_std, d_std, s_std, box_p))) return rc;
        const cuuint64_t d_yf[3] = {2 * ny, nx, nz}, s_yf[2] = {2 * ny * 4, 2 * nx * ny * 4};
        if ((rc = encode_one(&out->acc_yf, F32, 3, acc_yf, d_yf, s_yf, box_p))) return rc;
    }
    return LM_OK;
}

int tma_zlen(const lm_grid* g)
{
    const int ncol = ((g->n[0] + TD - 1) / TD) * ((g->n[1] + TD - 1) / TD);
    int nch = std::max(1, 2 * num_sms() / ncol);
    nch = std::min(nch, g->n[2]);
    return (g->n[2] + nch - 1) / nch;
}

int64_t tma_items_host(const lm_grid* g, int zlen)
{
    const int ncol = ((g->n[0] + TD - 1) / TD) * ((g->n[1] + TD - 1) / TD);
    return (int64_t)ncol * ((g->n[2] + zlen - 1) / zlen);
}

void launch_image_tma(const ImgArgs& a, cudaStream_t st)
{
    tma_attributes();
    lm_grid g;
    std::memset(&g, 0, sizeof(g));
    for (int d = 0; d < 3; ++d) g.n[d] = a.n[d];
    const int64_t items = tma_items_host(&g, a.zlen);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, 2 * (int64_t)num_sms()));
    image_tma_kernel<<<grid, 256, TmaLayout::total, st>>>(a);
    count_launch();
}

void launch_image_tma_batch(const BatchImgArgs& b, int grid, cudaStream_t st)
{
    tma_attributes();
    image_tma_batch_kernel<<<grid, 256, TmaLayout::total, st>>>(b);
    count_launch();
}

int image_tma_batch_grid(const lm_grid* g, int cap)
{
    const int64_t items = tma_items_host(g, tma_zlen(g)) * cap;
    return (int)std::max<int64_t>(1, std::min<int64_t>(items, 2 * (int64_t)num_sms()));
}

void launch_image_batch(const BatchImgArgs& b, int grid, cudaStream_t st)
{
    image_batch_kernel<<<grid, dim3(TD, TR), 0, st>>>(b);
    count_launch();
}

void launch_wpar_batch(const BatchImgArgs& b, int count, cudaStream_t st)
{
    wpar_batch_kernel<<<(b.cap + 63) / 64, 64, 0, st>>>(b, count);
    count_launch();
}

int image_batch_grid(const lm_grid* g, int cap)
{
    const int64_t nt = (int64_t)((g->n[0] + TD - 1) / TD) * ((g->n[1] + TD - 1) / TD) * g->n[2] * cap;
    return (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)num_sms() * 8));
}

int64_t image_tiles(const lm_grid* g)
{
    return (int64_t)((g->n[0] + TD - 1) / TD) * ((g->n[1] + TD - 1) / TD) * g->n[2];
}

void launch_wpar(const uint16_t* seq, int count, int n_subsets, int* wpar, int* wbase, cudaStream_t st)
{
    wpar_kernel<<<1, 32, 0, st>>>(seq, count, n_subsets, wpar, wbase);
    count_launch();
}

void launch_step_T(const lm_grid* g, const float* sens, float* T, float rho, float gamma, double knorm, int n_subsets,
                   cudaStream_t st)
{
    // T_k = gamma^-1 rho p_k / (P^T 1 / n) with p_k = 1/(2n): rho / (2 gamma sens)
    // T_{n+1} = gamma^-1 p_{n+1} rho / ||K|| with p_{n+1} = 1/2
    const double p_data = 1.0 / (2.0 * n_subsets), p_prior = 0.5;
    const float c_data = (float)((double)rho * p_data * n_subsets / (double)gamma);
    const float t_prior = (float)((double)rho * p_prior / ((double)gamma * knorm));
    const int64_t V = nvox(g);
    step_T_kernel<<<flat_grid(V), 256, 0, st>>>(sens, T, V, t_prior, c_data);
    count_launch();
}

int reduce_minmax(const float* x, int64_t n, float* dev_scratch, float* mn, float* mx, cudaStream_t st)
{
    minmax_partial<<<RB, 256, 0, st>>>(x, n, dev_scratch);
    minmax_final<<<1, 256, 0, st>>>(dev_scratch);
    count_launch(2);
    float h[2];
    LM_CUDA(cudaMemcpyAsync(h, dev_scratch + 2 * RB, 2 * sizeof(float), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    *mn = h[0];
    *mx = h[1];
    return LM_OK;
}

size_t objective_scratch_bytes() { return align_up((4 * RB + 4) * sizeof(double)); }

int objective_parts(const lm_grid* g, const float* sens, const float* x, const float* xi, const float* p,
                    const float* contam, float s_flat, const uint16_t* w, int64_t n_ev, double* scratch,
                    double* out4, cudaStream_t st)
{
    obj_img_partial<<<RB, 256, 0, st>>>(sens, x, xi, g->n[0], g->n[1], g->n[2], scratch);
    obj_ev_partial<<<RB, 256, 0, st>>>(p, contam, s_flat, w, n_ev, scratch);
    obj_final<<<1, 256, 0, st>>>(scratch);
    count_launch(3);
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(out4, scratch + 4 * RB, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    return LM_OK;
}

void launch_zadd(const lm_grid* g, const float* z, const float* zc, float* out, cudaStream_t st)
{
    const int64_t V = nvox(g);
    zadd_kernel<<<flat_grid(V), 256, 0, st>>>(z, zc, out, V);
    count_launch();
}

}  // namespace lmh

using namespace lmh;

extern "C" {

int lm_tv_ndim(const lm_grid* grid)
{
    if (check_grid(grid)) return -1;
    return tv_ndim(grid);
}

int lm_tv_grad(const lm_grid* grid, const float* x, float* g, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(x && g, LM_ERR_INVALID_ARG, "x or g is NULL");
    const int64_t V = nvox(grid);
    tv_grad_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(x, g, grid->n[0], grid->n[1], grid->n[2]);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lm_tv_div(const lm_grid* grid, const float* g, float* d, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(g && d, LM_ERR_INVALID_ARG, "g or d is NULL");
    const int64_t V = nvox(grid);
    tv_div_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(g, d, grid->n[0], grid->n[1], grid->n[2]);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lm_dtv_field(const lm_grid* grid, const float* v, float eta, float* xi, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(v && xi, LM_ERR_INVALID_ARG, "v or xi is NULL");
    LM_CHECK(eta >= 0.0f && std::isfinite(eta), LM_ERR_INVALID_ARG, "eta must be finite and >= 0");
    const int64_t V = nvox(grid);
    dtv_field_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(v, eta * eta, xi, grid->n[0], grid->n[1], grid->n[2]);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lm_dtv_grad(const lm_grid* grid, const float* xi, const float* x, float* g, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(xi && x && g, LM_ERR_INVALID_ARG, "xi, x or g is NULL");
    const int64_t V = nvox(grid);
    dtv_grad_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(x, xi, g, grid->n[0], grid->n[1], grid->n[2]);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lm_dtv_div(const lm_grid* grid, const float* xi, const float* g, float* d, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(xi && g && d, LM_ERR_INVALID_ARG, "xi, g or d is NULL");
    const int64_t V = nvox(grid);
    dtv_div_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(g, xi, d, grid->n[0], grid->n[1], grid->n[2]);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lm_tv_prox(const lm_grid* grid, float* w, float beta, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(w != nullptr, LM_ERR_INVALID_ARG, "w is NULL");
    LM_CHECK(beta >= 0.0f && std::isfinite(beta), LM_ERR_INVALID_ARG, "beta must be >= 0");
    const int64_t V = nvox(grid);
    tv_prox_kernel<<<flat_grid(V), 256, 0, S(stream)>>>(w, V, tv_ndim(grid), beta);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}


size_t lm_knorm_workspace_bytes(const lm_grid* grid)
{
    if (check_grid(grid)) return 0;
    const size_t V = (size_t)nvox(grid);
    return 2 * align_up(V * 8) + align_up((3 * RB + 8) * 8);
}

int lm_knorm_fp64(const lm_grid* grid, int32_t iters, void* ws, size_t ws_bytes, double* out_host, void* stream)
{
    clear_error();
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(out_host != nullptr, LM_ERR_INVALID_ARG, "out_host is NULL");
    LM_CHECK(iters >= 1, LM_ERR_INVALID_ARG, "iters must be >= 1");
    const size_t need = lm_knorm_workspace_bytes(grid);
    LM_CHECK(ws != nullptr && ws_bytes >= need, LM_ERR_NOMEM, "knorm needs %zu workspace bytes", need);
    cudaStream_t st = S(stream);
    const size_t V = (size_t)nvox(grid);
    char* w = (char*)ws;
    double* buf[2] = {(double*)w, (double*)(w + align_up(V * 8))};
    double* part = (double*)(w + 2 * align_up(V * 8));
    double* scal = part + 3 * RB;
    if (tv_ndim(grid) == 0) {
        *out_host = 0.0;
        return LM_OK;
    }
    kn_init<<<flat_grid((int64_t)V), 256, 0, st>>>(buf[0], grid->n[0], grid->n[1], grid->n[2]);
    const double one = 1.0;
    LM_CUDA(cudaMemcpyAsync(scal, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    for (int k = 0; k < iters; ++k) {
        kn_apply<<<RB, 256, 0, st>>>(buf[k & 1], buf[(k + 1) & 1], scal, grid->n[0], grid->n[1], grid->n[2], part);
        kn_final<<<1, 256, 0, st>>>(part, scal);
    }
    count_launch(1 + 2 * (int64_t)iters);
    LM_CUDA(cudaGetLastError());
    double lam = 0.0;
    LM_CUDA(cudaMemcpyAsync(&lam, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    *out_host = std::sqrt(lam);
    return LM_OK;
}

}  // extern "C"
