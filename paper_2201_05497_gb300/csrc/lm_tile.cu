// Tile-binned projector for the data updates of Alg. 2 (lines 10-13).
//
// The direct event kernel gathers and scatters each event's samples straight
// from/to L2; its atomics land on scattered sectors (a 32-lane request covers
// ~15 sectors), which bounds it by L2 atomic throughput.  Here the traversal
// of every event (its TOF window, Sec. "Listmode SPDHG"'s Joseph projector)
// is cut once per frame into segments: maximal runs of consecutive planes
// whose base voxel lies in one 32 x 32 x 8 image tile.  Segments are sorted
// by tile (and by subset), so a data update becomes
//   1. tl_fwd:  per work item (<= TL_CH segments of one tile) the tile of x
//               plus a one-voxel halo is loaded into shared memory and each
//               segment's partial forward projection is written to its slot;
//   2. tl_dual: per event, the partials of its segments are summed in segment
//               order (deterministic), then the dual step of Eq. (proxD);
//   3. tl_back: per work item, the back-projection of c_e v_e is accumulated
//               in a shared-memory tile and added to the image accumulator
//               once per tile voxel.
// Per sample the arithmetic is the direct kernel's (same positions, TOF
// table, bilinear weights, skip of zero weights); only the order of the sums
// differs.  (P^LM 1)_e, which S_e needs, is also computed once per frame.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lm_internal.h"

using namespace lmk;
using lmh::TileArgs;
using lmh::TileItem;

namespace {

constexpr int TX = lmh::TL_TX, TY = lmh::TL_TY;
constexpr int BXW = 36;  // shared tile row pitch (33 used: tile + halo)
constexpr int BYH = 33;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Stored traversal of one event: (ua0, sa, ub0, sb), (tau0, dtau, step, info)
// with info = k | 4 (valid) | i0 << 3 | cnt << 17.  Every later pass works
// from these stored values, so all of them cut and sample the traversal
// identically.
__device__ __forceinline__ int info_k(int info) { return info & 3; }
__device__ __forceinline__ int info_i0(int info) { return (info >> 3) & 0x3FFF; }
__device__ __forceinline__ int info_cnt(int info) { return (info >> 17) & 0x3FFF; }

// Tile of the (clamped) base voxel of plane i.
__device__ __forceinline__ int tile_of_plane(const TileArgs& A, const float4& e0, int k, bool two_d, int i)
{
    const float fi = (float)i;
    const int nA = k == 0 ? A.G.n[1] : A.G.n[0];
    const int nB = k == 2 ? A.G.n[1] : A.G.n[2];
    const int ia = clampi((int)floorf(fmaf(fi, e0.y, e0.x)), 0, nA - 1);
    const int ib = two_d ? 0 : clampi((int)floorf(fmaf(fi, e0.w, e0.z)), 0, nB - 1);
    const int c0 = k == 0 ? i : ia;
    const int c1 = k == 1 ? i : (k == 0 ? ia : ib);
    const int c2 = k == 2 ? i : ib;
    return ((c2 / A.tz) * A.ntile[1] + c1 / TY) * A.ntile[0] + c0 / TX;
}

// Subset of event q (events are subset-contiguous).
__device__ __forceinline__ int subset_of(const int64_t* sub_off, int n, int64_t q)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sub_off[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_tab(const float* g, float* s)
{
    for (int k = threadIdx.x; k <= lmh::TOF_TAB_N; k += blockDim.x) s[k] = g[k];
}

// Per event: traversal parameters, (P^LM 1)_e = c_e sum of sample weights,
// number of segments, and per (subset, tile) segment counts.
template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_count_kernel(const TileArgs A, int64_t N, unsigned* nseg_out,
                                                       unsigned* tile_cnt)
{
    extern __shared__ float s_tab[];
    load_tab(A.tof_tab, s_tab);
    __syncthreads();
    const Geo& G = A.G;
    const float inv_dt = (float)lmh::TOF_TAB_N / (2.0f * G.W);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const int d1 = A.det1[q], d2 = A.det2[q];
        const int m = (int)A.tofb[q];
        Lor L;
        bool ok = d1 >= 0 && d1 < G.n_det && d2 >= 0 && d2 < G.n_det && d1 != d2 && m >= -G.M && m <= G.M;
        ok = ok && lor_setup(G, d1, d2, m, TOF_BIN, false, L);
        float4 e0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), e1 = e0;
        unsigned ns = 0;
        float wsum_all = 0.0f;
        if (ok) {
            e0 = make_float4(L.ua0, L.sa, L.ub0, L.sb);
            e1 = make_float4(L.tau0, L.dtau, L.step, __int_as_float(L.k | 4 | (L.i0 << 3) | (L.cnt << 17)));
            const int sub = subset_of(A.sub_off, A.n_subsets, q);
            int cur = -1;
            for (int i = L.i0; i < L.i0 + L.cnt; ++i) {
                const float fi = (float)i;
                const float wt = L.step * lmh::tof_weight_tab(G, s_tab, inv_dt, fmaf(fi, L.dtau, L.tau0));
                if (wt != 0.0f) {
                    const float ua = fmaf(fi, L.sa, L.ua0);
                    const float fla = floorf(ua);
                    const int ia = (int)fla;
                    const float fa = ua - fla;
                    const float wa0 = (ia >= 0 && ia < L.nA) ? (1.0f - fa) : 0.0f;
                    const float wa1 = (ia + 1 >= 0 && ia + 1 < L.nA) ? fa : 0.0f;
                    if (TWO_D) {
                        wsum_all += wt * wa0 + wt * wa1;
                    } else {
                        const float ub = fmaf(fi, L.sb, L.ub0);
                        const float flb = floorf(ub);
                        const int ib = (int)flb;
                        const float fb = ub - flb;
                        const float wb0 = (ib >= 0 && ib < L.nB) ? (1.0f - fb) : 0.0f;
                        const float wb1 = (ib + 1 >= 0 && ib + 1 < L.nB) ? fb : 0.0f;
                        const float wA0 = wt * wa0, wA1 = wt * wa1;
                        wsum_all += (wA0 * wb0 + wA1 * wb0) + (wA0 * wb1 + wA1 * wb1);
                    }
                }
                const int t = tile_of_plane(A, e0, L.k, TWO_D, i);
                if (t != cur) {
                    atomicAdd(tile_cnt + (size_t)sub * A.n_tiles + t, 1u);
                    ++ns;
                    cur = t;
                }
            }
        }
        A.evp[2 * q] = e0;
        A.evp[2 * q + 1] = e1;
        A.p1[q] = ok ? (A.corr ? A.corr[q] : 1.0f) * wsum_all : 0.0f;
        nseg_out[q] = ns;
    }
}

// Segment records at their tile-sorted positions.
template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_fill_kernel(const TileArgs A, int64_t N, const unsigned* tile_off,
                                                      unsigned* tile_fill, unsigned total)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const float4 e1 = A.evp[2 * q + 1];
        const int info = __float_as_int(e1.w);
        if (!(info & 4)) continue;
        const float4 e0 = A.evp[2 * q];
        const int k = info_k(info), i0 = info_i0(info), iend = i0 + info_cnt(info);
        const int sub = subset_of(A.sub_off, A.n_subsets, q);
        const unsigned base = A.seg_off[q], lim = A.seg_off[q + 1];
        unsigned s = 0;
        int cur = -1, start = i0;
        for (int i = i0; i <= iend; ++i) {
            const int t = i < iend ? tile_of_plane(A, e0, k, TWO_D, i) : -2;
            if (t != cur) {
                if (cur >= 0) {
                    const size_t ti = (size_t)sub * A.n_tiles + cur;
                    const unsigned pos = tile_off[ti] + atomicAdd(tile_fill + ti, 1u);
                    // the enumeration is the count pass's; the checks only guard the buffers
                    if (pos < total && base + s < lim) {
                        A.seg[pos] = make_uint2((unsigned)q, (unsigned)start | ((unsigned)(i - start) << 16));
                        A.seg_pos[base + s] = pos;
                    }
                    ++s;
                }
                cur = t;
                start = i;
            }
        }
    }
}

// Exclusive scan helpers (set-up only): sums of blocks of SB elements, then
// the scan inside each block plus the (host-scanned) block offsets.
constexpr int SB = 2048;

__global__ void __launch_bounds__(256) tl_block_sums(const unsigned* v, int64_t n, unsigned long long* bs)
{
    __shared__ unsigned long long red[256];
    const int64_t b0 = (int64_t)blockIdx.x * SB;
    unsigned long long s = 0;
    for (int k = threadIdx.x; k < SB; k += 256)
        if (b0 + k < n) s += v[b0 + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) bs[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) tl_block_scan(const unsigned* v, int64_t n, const unsigned long long* boff,
                                                     unsigned* out)
{
    __shared__ unsigned long long part[256];
    const int64_t b0 = (int64_t)blockIdx.x * SB;
    constexpr int PER = SB / 256;
    unsigned loc[PER];
    unsigned long long s = 0;
    for (int k = 0; k < PER; ++k) {
        const int64_t idx = b0 + threadIdx.x * PER + k;
        loc[k] = idx < n ? v[idx] : 0u;
        s += loc[k];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = boff[blockIdx.x];
        for (int t = 0; t < 256; ++t) {
            const unsigned long long x = part[t];
            part[t] = run;
            run += x;
        }
    }
    __syncthreads();
    unsigned long long run = part[threadIdx.x];
    for (int k = 0; k < PER; ++k) {
        const int64_t idx = b0 + threadIdx.x * PER + k;
        if (idx < n) out[idx] = (unsigned)run;
        run += loc[k];
    }
}

// Origin of a tile and the depth of its shared-memory copy (tile + halo).
struct TileBox {
    int o0, o1, o2;
    int bz;
};

__device__ __forceinline__ TileBox box_of(const TileArgs& A, int tile)
{
    TileBox b;
    b.o0 = (tile % A.ntile[0]) * TX;
    b.o1 = ((tile / A.ntile[0]) % A.ntile[1]) * TY;
    b.o2 = (tile / (A.ntile[0] * A.ntile[1])) * A.tz;
    b.bz = A.G.n[2] > 1 ? A.tz + 1 : 1;
    return b;
}

// A segment's traversal in shared-tile coordinates: strides of the plane
// index and the two secondary axes and the offset of the tile origin.
struct SegFrame {
    int sk, sA, sB, off;
    int nA, nB;
};

__device__ __forceinline__ SegFrame seg_frame(const Geo& G, const TileBox& b, int k)
{
    constexpr int S1 = BXW, S2 = BXW * BYH;
    SegFrame f;
    // principal axis k, secondary A = (k == 0 ? y : x), B = (k == 2 ? y : z)
    f.sk = k == 0 ? 1 : (k == 1 ? S1 : S2);
    f.sA = k == 0 ? S1 : 1;
    f.sB = k == 2 ? S1 : S2;
    const int ok = k == 0 ? b.o0 : (k == 1 ? b.o1 : b.o2);
    const int oA = k == 0 ? b.o1 : b.o0;
    const int oB = k == 2 ? b.o1 : b.o2;
    f.off = -(ok * f.sk + oA * f.sA + oB * f.sB);
    f.nA = k == 0 ? G.n[1] : G.n[0];
    f.nB = k == 2 ? G.n[1] : G.n[2];
    return f;
}

// Loads the tile of x plus its +1 halo into shared memory (0 outside the grid).
__device__ __forceinline__ void load_box(const TileArgs& A, const TileBox& b, float* box)
{
    const int nx = A.G.n[0], ny = A.G.n[1], nz = A.G.n[2];
    const int rows = BYH * b.bz;
    for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5) {
        const int ly = r % BYH, lz = r / BYH;
        const int gy = b.o1 + ly, gz = b.o2 + lz;
        const bool rowin = gy < ny && gz < nz;
        for (int lx = threadIdx.x & 31; lx < BYH; lx += 32) {
            const int gx = b.o0 + lx;
            box[(lz * BYH + ly) * BXW + lx] =
                (rowin && gx < nx) ? __ldg(A.x + ((int64_t)gz * ny + gy) * nx + gx) : 0.0f;
        }
    }
}

// Sample of plane i of a segment in shared-tile coordinates: base offset and
// bilinear weights times TOF weight times step (the direct kernel's
// sample_tab, with the image strides replaced by the tile's).
struct TSmp {
    int base;
    float w0, w1, w2, w3;
};

template <bool TWO_D>
__device__ __forceinline__ bool tile_sample(const Geo& G, const float* tab, float inv_dt, const float4& e0,
                                            const float4& e1, const SegFrame& f, int i, TSmp& s)
{
    const float fi = (float)i;
    const float wt = e1.z * lmh::tof_weight_tab(G, tab, inv_dt, fmaf(fi, e1.y, e1.x));
    if (wt == 0.0f) return false;
    const float ua = fmaf(fi, e0.y, e0.x);
    const float fla = floorf(ua);
    const int ia = (int)fla;
    const float fa = ua - fla;
    const float wa0 = (ia >= 0 && ia < f.nA) ? (1.0f - fa) : 0.0f;
    const float wa1 = (ia + 1 >= 0 && ia + 1 < f.nA) ? fa : 0.0f;
    if (TWO_D) {
        s.base = i * f.sk + ia * f.sA + f.off;
        s.w0 = wt * wa0;
        s.w1 = wt * wa1;
        s.w2 = s.w3 = 0.0f;
        return (wa0 != 0.0f) || (wa1 != 0.0f);
    }
    const float ub = fmaf(fi, e0.w, e0.z);
    const float flb = floorf(ub);
    const int ib = (int)flb;
    const float fb = ub - flb;
    const float wb0 = (ib >= 0 && ib < f.nB) ? (1.0f - fb) : 0.0f;
    const float wb1 = (ib + 1 >= 0 && ib + 1 < f.nB) ? fb : 0.0f;
    s.base = i * f.sk + ia * f.sA + ib * f.sB + f.off;
    const float wA0 = wt * wa0, wA1 = wt * wa1;
    s.w0 = wA0 * wb0;
    s.w1 = wA1 * wb0;
    s.w2 = wA0 * wb1;
    s.w3 = wA1 * wb1;
    return (s.w0 != 0.0f) || (s.w1 != 0.0f) || (s.w2 != 0.0f) || (s.w3 != 0.0f);
}

constexpr int GL = 16;  // lanes per segment

template <bool TWO_D, bool BACK>
__device__ __forceinline__ void tile_segments(const TileArgs& A, const TileItem& I, const TileBox& b, float* box,
                                              const float* tab, float inv_dt)
{
    const Geo& G = A.G;
    const int lane = threadIdx.x & 31;
    const int sub = lane % GL;
    const int grp = threadIdx.x / GL, ngrp = blockDim.x / GL;
    const unsigned end = I.start + (unsigned)I.count;
    // every group runs the same number of rounds so the shuffles stay full-warp
    const int rounds = (I.count + ngrp - 1) / ngrp;
    for (int r = 0; r < rounds; ++r) {
        const unsigned j = I.start + (unsigned)(r * ngrp + grp);
        const bool have = j < end;
        uint2 sg = make_uint2(0u, 0u);
        if (have) sg = __ldg(A.seg + j);
        const unsigned q = sg.x;
        const int i_a = (int)(sg.y & 0xFFFFu), len = have ? (int)(sg.y >> 16) : 0;
        float4 e0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), e1 = e0;
        float bv = 0.0f;
        if (have) {
            e0 = __ldg(A.evp + 2 * (size_t)q);
            e1 = __ldg(A.evp + 2 * (size_t)q + 1);
            if (BACK) bv = A.v[q];
        }
        const SegFrame f = seg_frame(G, b, __float_as_int(e1.w) & 3);
        float acc = 0.0f;
        if (!BACK || bv != 0.0f) {
            for (int p = sub; p < len; p += GL) {
                TSmp s;
                if (!tile_sample<TWO_D>(G, tab, inv_dt, e0, e1, f, i_a + p, s)) continue;
                if (BACK) {
                    if (s.w0 != 0.0f) atomicAdd(box + s.base, s.w0 * bv);
                    if (s.w1 != 0.0f) atomicAdd(box + s.base + f.sA, s.w1 * bv);
                    if (!TWO_D) {
                        if (s.w2 != 0.0f) atomicAdd(box + s.base + f.sB, s.w2 * bv);
                        if (s.w3 != 0.0f) atomicAdd(box + s.base + f.sA + f.sB, s.w3 * bv);
                    }
                } else {
                    if (s.w0 != 0.0f) acc = fmaf(s.w0, box[s.base], acc);
                    if (s.w1 != 0.0f) acc = fmaf(s.w1, box[s.base + f.sA], acc);
                    if (!TWO_D) {
                        if (s.w2 != 0.0f) acc = fmaf(s.w2, box[s.base + f.sB], acc);
                        if (s.w3 != 0.0f) acc = fmaf(s.w3, box[s.base + f.sA + f.sB], acc);
                    }
                }
            }
        }
        if (!BACK) {
#pragma unroll
            for (int o = GL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o, GL);
            if (have && sub == 0) A.part[j] = acc;
        }
    }
}

__device__ __forceinline__ bool prior_selected(const TileArgs& A, int& sel)
{
    sel = A.seq[A.u];
    return sel >= A.n_subsets;
}

template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_fwd_kernel(const TileArgs A)
{
    int sel;
    if (prior_selected(A, sel)) return;
    extern __shared__ float smem[];
    float* tab = smem;
    float* box = smem + (lmh::TOF_TAB_N + 4);
    load_tab(A.tof_tab, tab);
    const float inv_dt = (float)lmh::TOF_TAB_N / (2.0f * A.G.W);
    const int i0 = A.item_off[sel], i1 = A.item_off[sel + 1];
    for (int it = i0 + blockIdx.x; it < i1; it += gridDim.x) {
        const TileItem I = A.items[it];
        const TileBox b = box_of(A, I.tile);
        __syncthreads();  // previous item done with the box (and the table is loaded)
        load_box(A, b, box);
        __syncthreads();
        tile_segments<TWO_D, false>(A, I, b, box, tab, inv_dt);
    }
}

// Dual step per event of the selected subset (Eq. proxD with mu S_e).
__global__ void __launch_bounds__(256) tl_dual_kernel(const TileArgs A)
{
    int sel;
    if (prior_selected(A, sel)) return;
    const int64_t e0 = A.sub_off[sel], e1 = A.sub_off[sel + 1];
    for (int64_t q = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < e1;
         q += (int64_t)gridDim.x * blockDim.x) {
        const unsigned a = A.seg_off[q], z = A.seg_off[q + 1];
        float J = 0.0f;
        for (unsigned s = a; s < z; ++s) J += A.part[A.seg_pos[s]];
        const float c = A.corr ? A.corr[q] : 1.0f;
        const float p1 = A.p1[q];
        const float y = A.y[q];
        const float mu = (float)A.mu[q];
        const float Se = p1 > 0.0f ? A.gamma_rho / p1 : 0.0f;
        const float aa = fmaf(Se, fmaf(c, J, A.contam[q]), y);
        const float yp = prox_dstar(aa, mu * Se);
        const float v = (yp - y) / mu;
        A.y[q] = yp;
        A.v[q] = z > a ? c * v : 0.0f;
    }
}

template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_back_kernel(const TileArgs A)
{
    int sel;
    if (prior_selected(A, sel)) return;
    extern __shared__ float smem[];
    float* tab = smem;
    float* box = smem + (lmh::TOF_TAB_N + 4);
    load_tab(A.tof_tab, tab);
    const float inv_dt = (float)lmh::TOF_TAB_N / (2.0f * A.G.W);
    const int nx = A.G.n[0], ny = A.G.n[1], nz = A.G.n[2];
    const int i0 = A.item_off[sel], i1 = A.item_off[sel + 1];
    for (int it = i0 + blockIdx.x; it < i1; it += gridDim.x) {
        const TileItem I = A.items[it];
        const TileBox b = box_of(A, I.tile);
        __syncthreads();
        for (int k = threadIdx.x; k < BXW * BYH * b.bz; k += blockDim.x) box[k] = 0.0f;
        __syncthreads();
        tile_segments<TWO_D, true>(A, I, b, box, tab, inv_dt);
        __syncthreads();
        const int rows = BYH * b.bz;
        for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5) {
            const int ly = r % BYH, lz = r / BYH;
            const int gy = b.o1 + ly, gz = b.o2 + lz;
            if (gy >= ny || gz >= nz) continue;
            for (int lx = threadIdx.x & 31; lx < BYH; lx += 32) {
                const int gx = b.o0 + lx;
                const float val = box[(lz * BYH + ly) * BXW + lx];
                if (gx < nx && val != 0.0f) atomicAdd(A.acc + ((int64_t)gz * ny + gy) * nx + gx, val);
            }
        }
    }
}

size_t tab_bytes() { return (size_t)(lmh::TOF_TAB_N + 1) * sizeof(float); }
size_t tile_smem(int bz) { return (size_t)(lmh::TOF_TAB_N + 4) * 4 + (size_t)BXW * BYH * bz * 4; }

}  // namespace

namespace lmh {

void tile_geometry(const lm_grid* g, int ntile[3], int* tz, int64_t* n_tiles)
{
    *tz = g->n[2] > 1 ? TL_TZ : 1;
    ntile[0] = (g->n[0] + TX - 1) / TX;
    ntile[1] = (g->n[1] + TY - 1) / TY;
    ntile[2] = (g->n[2] + *tz - 1) / *tz;
    *n_tiles = (int64_t)ntile[0] * ntile[1] * ntile[2];
}

TileLayout tile_layout(const lm_grid* g, int64_t N, int n_subsets)
{
    int nt[3], tz;
    int64_t ntiles;
    tile_geometry(g, nt, &tz, &ntiles);
    TileLayout L;
    const int64_t cap = TL_SEGCAP * std::max<int64_t>(N, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.cap = cap;
    L.max_items = (int64_t)n_subsets * ntiles + cap / TL_CH + n_subsets + 1;
    L.evp = take((size_t)std::max<int64_t>(N, 1) * 32);
    L.p1 = take((size_t)std::max<int64_t>(N, 1) * 4);
    L.seg_off = take((size_t)(N + 1) * 4);
    L.nseg = take((size_t)std::max<int64_t>(N, 1) * 4);
    L.seg = take((size_t)cap * 8);
    L.seg_pos = take((size_t)cap * 4);
    L.part = take((size_t)cap * 4);
    L.tiles = take((size_t)n_subsets * ntiles * 4 * 3);
    L.items = take((size_t)L.max_items * sizeof(TileItem));
    L.item_off = take((size_t)(n_subsets + 1) * 4);
    L.bsums = take((size_t)((N + SB) / SB + 1) * 8);
    L.total = off + 256;
    return L;
}

int tile_build(TileArgs& A, const TileLayout& Lt, char* base, int64_t N, const std::vector<int64_t>& sub_off_h,
               bool two_d, cudaStream_t st, int64_t* n_segments)
{
    const int n = A.n_subsets;
    const int64_t nt = A.n_tiles;
    unsigned* tile_cnt = (unsigned*)(base + Lt.tiles);
    unsigned* tile_off = tile_cnt + (size_t)n * nt;
    unsigned* tile_fill = tile_off + (size_t)n * nt;
    unsigned* nseg = (unsigned*)(base + Lt.nseg);
    unsigned long long* bsums = (unsigned long long*)(base + Lt.bsums);
    *n_segments = 0;
    LM_CUDA(cudaMemsetAsync(tile_cnt, 0, (size_t)n * nt * 4 * 3, st));
    if (N == 0) {
        std::vector<int> io(n + 1, 0);
        LM_CUDA(cudaMemcpyAsync(A.item_off, io.data(), io.size() * 4, cudaMemcpyHostToDevice, st));
        LM_CUDA(cudaMemsetAsync(A.seg_off, 0, 4, st));
        LM_CUDA(cudaStreamSynchronize(st));
        return LM_OK;
    }
    const int grid = (int)std::min<int64_t>((N + 255) / 256, (int64_t)num_sms() * 16);
    if (two_d) tl_count_kernel<true><<<grid, 256, tab_bytes(), st>>>(A, N, nseg, tile_cnt);
    else tl_count_kernel<false><<<grid, 256, tab_bytes(), st>>>(A, N, nseg, tile_cnt);
    count_launch();
    const int64_t nb = (N + SB - 1) / SB;
    tl_block_sums<<<(int)nb, 256, 0, st>>>(nseg, N, bsums);
    count_launch();
    std::vector<unsigned long long> hb((size_t)nb);
    LM_CUDA(cudaMemcpyAsync(hb.data(), bsums, (size_t)nb * 8, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    unsigned long long run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const unsigned long long x = hb[b];
        hb[b] = run;
        run += x;
    }
    *n_segments = (int64_t)run;
    LM_CHECK(run <= (unsigned long long)Lt.cap && run < (1ull << 32), LM_ERR_NOMEM,
             "tile binning needs %llu segments, capacity %lld", run, (long long)Lt.cap);
    LM_CUDA(cudaMemcpyAsync(bsums, hb.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, st));
    tl_block_scan<<<(int)nb, 256, 0, st>>>(nseg, N, bsums, A.seg_off);
    count_launch();
    const unsigned total = (unsigned)run;
    LM_CUDA(cudaMemcpyAsync(A.seg_off + N, &total, 4, cudaMemcpyHostToDevice, st));
    // per-subset tile offsets (segments of subset k occupy [seg_off[sub_off[k]], seg_off[sub_off[k+1]]))
    std::vector<unsigned> hc((size_t)n * nt), ho((size_t)n * nt);
    std::vector<unsigned> base_k(n + 1);
    LM_CUDA(cudaMemcpyAsync(hc.data(), tile_cnt, hc.size() * 4, cudaMemcpyDeviceToHost, st));
    for (int k = 0; k <= n; ++k)
        LM_CUDA(cudaMemcpyAsync(&base_k[k], A.seg_off + sub_off_h[k], 4, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    std::vector<TileItem> items;
    std::vector<int> io(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        io[k] = (int)items.size();
        unsigned pos = base_k[k];
        for (int64_t t = 0; t < nt; ++t) {
            const unsigned c = hc[(size_t)k * nt + t];
            ho[(size_t)k * nt + t] = pos;
            for (unsigned s0 = 0; s0 < c; s0 += TL_CH) {
                TileItem it;
                it.tile = (int)t;
                it.start = pos + s0;
                it.count = (int)std::min<unsigned>(TL_CH, c - s0);
                it.pad = 0;
                items.push_back(it);
            }
            pos += c;
        }
    }
    io[n] = (int)items.size();
    LM_CHECK((int64_t)items.size() <= Lt.max_items, LM_ERR_NOMEM, "tile work items exceed capacity");
    LM_CUDA(cudaMemcpyAsync(tile_off, ho.data(), ho.size() * 4, cudaMemcpyHostToDevice, st));
    if (!items.empty())
        LM_CUDA(cudaMemcpyAsync(A.items, items.data(), items.size() * sizeof(TileItem), cudaMemcpyHostToDevice,
                                st));
    LM_CUDA(cudaMemcpyAsync(A.item_off, io.data(), io.size() * 4, cudaMemcpyHostToDevice, st));
    if (two_d) tl_fill_kernel<true><<<grid, 256, 0, st>>>(A, N, tile_off, tile_fill, total);
    else tl_fill_kernel<false><<<grid, 256, 0, st>>>(A, N, tile_off, tile_fill, total);
    count_launch();
    int max_items = 0;
    for (int k = 0; k < n; ++k) max_items = std::max(max_items, io[k + 1] - io[k]);
    A.max_items = max_items;
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

void tile_attributes()
{
    static bool done = false;
    if (done) return;
    const size_t sm = tile_smem(TL_TZ + 1);
    cudaFuncSetAttribute(tl_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(tl_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(tl_back_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(tl_back_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    done = true;
}

int launch_tile_update(const TileArgs& A, bool two_d, cudaStream_t st)
{
    const size_t sm = tile_smem(A.G.n[2] > 1 ? A.tz + 1 : 1);
    const int g_tile = std::max(1, std::min(A.max_items, 3 * num_sms()));
    if (two_d) tl_fwd_kernel<true><<<g_tile, 256, sm, st>>>(A);
    else tl_fwd_kernel<false><<<g_tile, 256, sm, st>>>(A);
    tl_dual_kernel<<<num_sms() * 8, 256, 0, st>>>(A);
    if (two_d) tl_back_kernel<true><<<g_tile, 256, sm, st>>>(A);
    else tl_back_kernel<false><<<g_tile, 256, sm, st>>>(A);
    count_launch(3);
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

}  // namespace lmh
