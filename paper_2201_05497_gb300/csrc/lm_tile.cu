// Tile-binned projector for the data updates of Alg. 2 (forward projection,
// dual step, back-projection of the dual change).
//
// The direct event kernel gathers and scatters each event's samples straight
// from/to L2; its atomics land on scattered sectors (a 32-lane request covers
// ~15 sectors), which bounds it by L2 atomic throughput.  Here the traversal
// of every event (its TOF window, the Joseph projector of Sec. "Listmode
// SPDHG") is cut once per frame into segments: maximal runs of consecutive
// planes whose base voxel lies in one 32 x 32 x 8 image tile.  Segments are
// sorted by (subset, tile), so a data update becomes
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
//
// Latency: a warp loads the records of 32 segments (or the set-up of 32
// events) at once, one per lane, and hands them to its two 16-lane halves by
// shuffles, so one round trip to L2 serves 32 segments.
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
constexpr int GL = 16;   // lanes per segment

struct BinBlock {
    long long e0, e1;
    int sub, pad;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Stored traversal of one event: (ua0, sa, ub0, sb), (tau0, dtau, step, info)
// with info = k | 4 (valid) | i0 << 3 | cnt << 17.  Every pass works from
// these stored values, so all of them cut and sample a traversal identically.
__device__ __forceinline__ int info_k(int info) { return info & 3; }
__device__ __forceinline__ int info_i0(int info) { return (info >> 3) & 0x3FFF; }
__device__ __forceinline__ int info_cnt(int info) { return (info >> 17) & 0x3FFF; }

// Tile of the (clamped) base voxel of plane i.
__device__ __forceinline__ int tile_of_plane(const TileArgs& A, float ua0, float sa, float ub0, float sb, int k,
                                             bool two_d, int i)
{
    const float fi = (float)i;
    const int nA = k == 0 ? A.G.n[1] : A.G.n[0];
    const int nB = k == 2 ? A.G.n[1] : A.G.n[2];
    const int ia = clampi((int)floorf(fmaf(fi, sa, ua0)), 0, nA - 1);
    const int ib = two_d ? 0 : clampi((int)floorf(fmaf(fi, sb, ub0)), 0, nB - 1);
    const int c0 = k == 0 ? i : ia;
    const int c1 = k == 1 ? i : (k == 0 ? ia : ib);
    const int c2 = k == 2 ? i : ib;
    return ((c2 / A.tz) * A.ntile[1] + c1 / TY) * A.ntile[0] + c0 / TX;
}

__device__ __forceinline__ void load_tab(const float* g, float* s)
{
    for (int k = threadIdx.x; k <= lmh::TOF_TAB_N; k += blockDim.x) s[k] = g[k];
}

// Shuffled copy of lane src's stored traversal.
struct Trav {
    float ua0, sa, ub0, sb, tau0, dtau, step;
    int info;
};

__device__ __forceinline__ Trav shfl_trav(const float4& e0, const float4& e1, int src)
{
    Trav t;
    t.ua0 = __shfl_sync(FULL, e0.x, src);
    t.sa = __shfl_sync(FULL, e0.y, src);
    t.ub0 = __shfl_sync(FULL, e0.z, src);
    t.sb = __shfl_sync(FULL, e0.w, src);
    t.tau0 = __shfl_sync(FULL, e1.x, src);
    t.dtau = __shfl_sync(FULL, e1.y, src);
    t.step = __shfl_sync(FULL, e1.z, src);
    t.info = __shfl_sync(FULL, __float_as_int(e1.w), src);
    return t;
}

// Walks the planes of one traversal with the whole warp (32 planes per pass)
// and calls seg(s, tile, first_plane, planes) once per segment, from one lane
// (s is the segment's index within the event).  Returns, on every lane, the
// number of segments.
template <class F>
__device__ __forceinline__ int warp_segments(const TileArgs& A, const Trav& t, bool two_d, F&& seg)
{
    const int lane = threadIdx.x & 31;
    const int k = info_k(t.info), i0 = info_i0(t.info), iend = i0 + info_cnt(t.info);
    int carry = -1, open_start = -1, open_t = -1, open_s = 0, ns = 0;
    for (int b = i0; b < iend; b += 32) {
        const int i = b + lane;
        const bool in = i < iend;
        const int tl = in ? tile_of_plane(A, t.ua0, t.sa, t.ub0, t.sb, k, two_d, i) : -2;
        int prev = __shfl_up_sync(FULL, tl, 1);
        if (lane == 0) prev = carry;
        const bool bnd = in && tl != prev;
        const unsigned mask = __ballot_sync(FULL, bnd);
        if (mask) {
            const int first = __ffs(mask) - 1;
            if (open_start >= 0 && lane == first) seg(open_s, open_t, open_start, i - open_start);
            if (bnd) {
                const unsigned above = mask & ~((2u << lane) - 1u);
                if (above) {
                    const int end = b + __ffs(above) - 1;
                    seg(ns + __popc(mask & ((1u << lane) - 1u)), tl, i, end - i);
                }
            }
            const int last = 31 - __clz(mask);
            open_start = __shfl_sync(FULL, i, last);
            open_t = __shfl_sync(FULL, tl, last);
            open_s = ns + __popc(mask) - 1;
            ns += __popc(mask);
        }
        carry = __shfl_sync(FULL, tl, 31);
    }
    if (open_start >= 0 && lane == 0) seg(open_s, open_t, open_start, iend - open_start);
    return ns;
}

// Per event: traversal parameters and (P^LM 1)_e = c_e sum of sample weights;
// per binning block: segment counts per tile (block histogram).
template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_count_kernel(const TileArgs A, const BinBlock* bb, unsigned* nseg_out,
                                                       unsigned* bhist)
{
    extern __shared__ float smem[];
    float* tab = smem;
    unsigned* hist = reinterpret_cast<unsigned*>(smem + lmh::TOF_TAB_N + 4);
    load_tab(A.tof_tab, tab);
    for (int k = threadIdx.x; k < A.n_tiles; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const Geo& G = A.G;
    const float inv_dt = (float)lmh::TOF_TAB_N / (2.0f * G.W);
    const BinBlock B = bb[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long e0 = B.e0 + 32LL * warp; e0 < B.e1; e0 += 32LL * nw) {
        // lane l sets up event e0 + l
        const long long q = e0 + lane;
        const bool have = q < B.e1;
        Lor L;
        bool ok = false;
        float c = 1.0f;
        if (have) {
            const int d1 = A.det1[q], d2 = A.det2[q];
            const int m = (int)A.tofb[q];
            if (A.corr) c = A.corr[q];
            ok = d1 >= 0 && d1 < G.n_det && d2 >= 0 && d2 < G.n_det && d1 != d2 && m >= -G.M && m <= G.M;
            ok = ok && lor_setup(G, d1, d2, m, TOF_BIN, false, L) && L.cnt < 16384 && L.i0 < 16384;
        }
        float4 e0v = make_float4(0.0f, 0.0f, 0.0f, 0.0f), e1v = e0v;
        if (ok) {
            e0v = make_float4(L.ua0, L.sa, L.ub0, L.sb);
            e1v = make_float4(L.tau0, L.dtau, L.step, __int_as_float(L.k | 4 | (L.i0 << 3) | (L.cnt << 17)));
        }
        if (have) {
            A.evp[2 * q] = e0v;
            A.evp[2 * q + 1] = e1v;
        }
        const int nev = (int)min(32LL, B.e1 - e0);
        float my_p1 = 0.0f;
        unsigned my_ns = 0;
        for (int r = 0; r < nev; ++r) {
            const Trav t = shfl_trav(e0v, e1v, r);
            if (!(t.info & 4)) continue;  // warp-uniform
            // sample weights of this lane's planes (the direct kernel's per-sample weights)
            const int k = info_k(t.info), i0 = info_i0(t.info), iend = i0 + info_cnt(t.info);
            const int nA = k == 0 ? G.n[1] : G.n[0];
            const int nB = k == 2 ? G.n[1] : G.n[2];
            float ws = 0.0f;
            for (int i = i0 + lane; i < iend; i += 32) {
                const float fi = (float)i;
                const float wt = t.step * lmh::tof_weight_tab(G, tab, inv_dt, fmaf(fi, t.dtau, t.tau0));
                if (wt == 0.0f) continue;
                const float ua = fmaf(fi, t.sa, t.ua0);
                const float fla = floorf(ua);
                const int ia = (int)fla;
                const float fa = ua - fla;
                const float wa0 = (ia >= 0 && ia < nA) ? (1.0f - fa) : 0.0f;
                const float wa1 = (ia + 1 >= 0 && ia + 1 < nA) ? fa : 0.0f;
                if (TWO_D) {
                    ws += wt * wa0 + wt * wa1;
                } else {
                    const float ub = fmaf(fi, t.sb, t.ub0);
                    const float flb = floorf(ub);
                    const int ib = (int)flb;
                    const float fb = ub - flb;
                    const float wb0 = (ib >= 0 && ib < nB) ? (1.0f - fb) : 0.0f;
                    const float wb1 = (ib + 1 >= 0 && ib + 1 < nB) ? fb : 0.0f;
                    const float wA0 = wt * wa0, wA1 = wt * wa1;
                    ws += (wA0 * wb0 + wA1 * wb0) + (wA0 * wb1 + wA1 * wb1);
                }
            }
            ws = warp_sum(ws);
            const int ns = warp_segments(A, t, TWO_D, [&](int, int tl, int, int) { atomicAdd(hist + tl, 1u); });
            if (lane == r) {
                my_p1 = ws;
                my_ns = (unsigned)ns;
            }
        }
        if (have) {
            A.p1[q] = ok ? c * my_p1 : 0.0f;
            nseg_out[q] = ok ? my_ns : 0u;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < A.n_tiles; k += blockDim.x) bhist[(size_t)blockIdx.x * A.n_tiles + k] = hist[k];
}

// Offsets of every binning block within its subset's tile ranges: for each
// (subset, tile), blocks in order.  Also the per-(subset, tile) totals.
__global__ void tl_block_offsets(const int* bsub_off, int n, int64_t n_tiles, unsigned* bhist, unsigned* tile_cnt)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)n * n_tiles) return;
    const int sub = (int)(id / n_tiles);
    const int64_t t = id - (int64_t)sub * n_tiles;
    unsigned run = 0;
    for (int b = bsub_off[sub]; b < bsub_off[sub + 1]; ++b) {
        unsigned* h = bhist + (size_t)b * n_tiles + t;
        const unsigned c = *h;
        *h = run;  // becomes the block's offset
        run += c;
    }
    tile_cnt[id] = run;
}

// Segment records at their tile-sorted positions.
template <bool TWO_D>
__global__ void __launch_bounds__(256) tl_fill_kernel(const TileArgs A, const BinBlock* bb, const unsigned* bhist,
                                                      const unsigned* tile_off, unsigned total)
{
    extern __shared__ unsigned s_u[];
    unsigned* base = s_u;
    unsigned* cnt = s_u + A.n_tiles;
    const BinBlock B = bb[blockIdx.x];
    for (int k = threadIdx.x; k < A.n_tiles; k += blockDim.x) {
        base[k] = tile_off[(size_t)B.sub * A.n_tiles + k] + bhist[(size_t)blockIdx.x * A.n_tiles + k];
        cnt[k] = 0u;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (long long e0 = B.e0 + 32LL * warp; e0 < B.e1; e0 += 32LL * nw) {
        const long long q = e0 + lane;
        float4 e0v = make_float4(0.0f, 0.0f, 0.0f, 0.0f), e1v = e0v;
        unsigned sbase = 0, slim = 0;
        if (q < B.e1) {
            e0v = A.evp[2 * q];
            e1v = A.evp[2 * q + 1];
            sbase = A.seg_off[q];
            slim = A.seg_off[q + 1];
        }
        const int nev = (int)min(32LL, B.e1 - e0);
        for (int r = 0; r < nev; ++r) {
            const Trav t = shfl_trav(e0v, e1v, r);
            const unsigned qb = __shfl_sync(FULL, sbase, r), ql = __shfl_sync(FULL, slim, r);
            if (!(t.info & 4)) continue;  // warp-uniform
            const unsigned qe = (unsigned)(e0 + r);
            warp_segments(A, t, TWO_D, [&](int s, int tl, int start, int len) {
                const unsigned pos = base[tl] + atomicAdd(cnt + tl, 1u);
                // the enumeration is the count pass's; the checks only guard the buffers
                if (pos < total && qb + (unsigned)s < ql) {
                    A.seg[pos] = make_uint2(qe, (unsigned)start | ((unsigned)len << 16));
                    A.seg_pos[qb + s] = pos;
                }
            });
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
__device__ __forceinline__ bool tile_sample(const Geo& G, const float* tab, float inv_dt, const Trav& t,
                                            const SegFrame& f, int i, TSmp& s)
{
    const float fi = (float)i;
    const float wt = t.step * lmh::tof_weight_tab(G, tab, inv_dt, fmaf(fi, t.dtau, t.tau0));
    if (wt == 0.0f) return false;
    const float ua = fmaf(fi, t.sa, t.ua0);
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
    const float ub = fmaf(fi, t.sb, t.ub0);
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

// The segments of one work item: each warp takes batches of 32 (one record
// per lane, loaded together), its two halves process two segments at a time.
template <bool TWO_D, bool BACK>
__device__ __forceinline__ void tile_segments(const TileArgs& A, const TileItem& I, const TileBox& b, float* box,
                                              const float* tab, float inv_dt)
{
    const Geo& G = A.G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int half = lane / GL, sub = lane % GL;
    const unsigned end = I.start + (unsigned)I.count;
    for (unsigned j0 = I.start + 32u * warp; j0 < end; j0 += 32u * nw) {
        const unsigned jl = j0 + lane;
        float4 e0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), e1 = e0;
        unsigned sy = 0;
        float bv = 0.0f;
        if (jl < end) {
            const uint2 sg = __ldg(A.seg + jl);
            sy = sg.y;
            e0 = __ldg(A.evp + 2 * (size_t)sg.x);
            e1 = __ldg(A.evp + 2 * (size_t)sg.x + 1);
            if (BACK) bv = A.v[sg.x];
        }
        const int nseg = (int)min(32u, end - j0);
        for (int r = 0; 2 * r < nseg; ++r) {
            const int src = 2 * r + half;
            const Trav t = shfl_trav(e0, e1, src);
            const unsigned sys = __shfl_sync(FULL, sy, src);
            const float bvs = BACK ? __shfl_sync(FULL, bv, src) : 0.0f;
            const bool valid = src < nseg;
            const int i_a = (int)(sys & 0xFFFFu), len = valid ? (int)(sys >> 16) : 0;
            const SegFrame f = seg_frame(G, b, info_k(t.info));
            float acc = 0.0f;
            if (!BACK || bvs != 0.0f) {
                for (int p = sub; p < len; p += GL) {
                    TSmp s;
                    if (!tile_sample<TWO_D>(G, tab, inv_dt, t, f, i_a + p, s)) continue;
                    if (BACK) {
                        if (s.w0 != 0.0f) atomicAdd(box + s.base, s.w0 * bvs);
                        if (s.w1 != 0.0f) atomicAdd(box + s.base + f.sA, s.w1 * bvs);
                        if (!TWO_D) {
                            if (s.w2 != 0.0f) atomicAdd(box + s.base + f.sB, s.w2 * bvs);
                            if (s.w3 != 0.0f) atomicAdd(box + s.base + f.sA + f.sB, s.w3 * bvs);
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
                if (valid && sub == 0) A.part[j0 + src] = acc;
            }
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
                // the accumulator holds z pairs: voxel j is element 2j
                if (gx < nx && val != 0.0f) atomicAdd(A.acc + 2 * (((int64_t)gz * ny + gy) * nx + gx), val);
            }
        }
    }
}

size_t tile_smem(int bz) { return (size_t)(lmh::TOF_TAB_N + 4) * 4 + (size_t)BXW * BYH * bz * 4; }
size_t count_smem(int64_t n_tiles) { return (size_t)(lmh::TOF_TAB_N + 4) * 4 + (size_t)n_tiles * 4; }

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
    L.max_bblocks = N / TL_EPB + n_subsets + 1;
    L.evp = take((size_t)std::max<int64_t>(N, 1) * 32);
    L.p1 = take((size_t)std::max<int64_t>(N, 1) * 4);
    L.seg_off = take((size_t)(N + 1) * 4);
    L.nseg = take((size_t)std::max<int64_t>(N, 1) * 4);
    L.seg = take((size_t)cap * 8);
    L.seg_pos = take((size_t)cap * 4);
    L.part = take((size_t)cap * 4);
    L.tiles = take((size_t)n_subsets * ntiles * 4 * 2);
    L.items = take((size_t)L.max_items * sizeof(TileItem));
    L.item_off = take((size_t)(n_subsets + 1) * 4);
    L.bsums = take((size_t)((N + SB) / SB + 1) * 8);
    L.bblocks = take((size_t)L.max_bblocks * sizeof(BinBlock) + (size_t)(n_subsets + 1) * 4);
    L.bhist = take((size_t)L.max_bblocks * ntiles * 4);
    L.total = off + 256;
    return L;
}

int tile_build(TileArgs& A, const TileLayout& Lt, char* base, int64_t N, const std::vector<int64_t>& sub_off_h,
               bool two_d, cudaStream_t st, int64_t* n_segments)
{
    const int n = A.n_subsets;
    const int64_t nt = A.n_tiles;
    *n_segments = 0;
    LM_CHECK(nt <= TL_MAX_TILES, LM_ERR_NOMEM, "tile grid of %lld tiles exceeds %d", (long long)nt, TL_MAX_TILES);
    unsigned* tile_cnt = (unsigned*)(base + Lt.tiles);
    unsigned* tile_off = tile_cnt + (size_t)n * nt;
    unsigned* nseg = (unsigned*)(base + Lt.nseg);
    unsigned long long* bsums = (unsigned long long*)(base + Lt.bsums);
    BinBlock* bb = (BinBlock*)(base + Lt.bblocks);
    int* bsub_off = (int*)(base + Lt.bblocks + (size_t)Lt.max_bblocks * sizeof(BinBlock));
    unsigned* bhist = (unsigned*)(base + Lt.bhist);
    // binning blocks: contiguous event ranges of at most TL_EPB inside one subset
    std::vector<BinBlock> hb;
    std::vector<int> hbo(n + 1, 0);
    for (int k = 0; k < n; ++k) {
        hbo[k] = (int)hb.size();
        for (int64_t e = sub_off_h[k]; e < sub_off_h[k + 1]; e += TL_EPB) {
            BinBlock b;
            b.e0 = e;
            b.e1 = std::min<int64_t>(sub_off_h[k + 1], e + TL_EPB);
            b.sub = k;
            b.pad = 0;
            hb.push_back(b);
        }
    }
    hbo[n] = (int)hb.size();
    LM_CHECK((int64_t)hb.size() <= Lt.max_bblocks, LM_ERR_NOMEM, "binning blocks exceed capacity");
    const int nbb = (int)hb.size();
    if (N == 0 || nbb == 0) {
        std::vector<int> io(n + 1, 0);
        LM_CUDA(cudaMemcpyAsync(A.item_off, io.data(), io.size() * 4, cudaMemcpyHostToDevice, st));
        LM_CUDA(cudaMemsetAsync(A.seg_off, 0, 4, st));
        A.max_items = 0;
        LM_CUDA(cudaStreamSynchronize(st));
        return LM_OK;
    }
    LM_CUDA(cudaMemcpyAsync(bb, hb.data(), hb.size() * sizeof(BinBlock), cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(bsub_off, hbo.data(), hbo.size() * 4, cudaMemcpyHostToDevice, st));
    const size_t csm = count_smem(nt);
    if (csm > 48 * 1024) {
        cudaFuncSetAttribute(tl_count_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
        cudaFuncSetAttribute(tl_count_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
    }
    if (two_d) tl_count_kernel<true><<<nbb, 256, csm, st>>>(A, bb, nseg, bhist);
    else tl_count_kernel<false><<<nbb, 256, csm, st>>>(A, bb, nseg, bhist);
    const int64_t nbo = (int64_t)n * nt;
    tl_block_offsets<<<(int)((nbo + 255) / 256), 256, 0, st>>>(bsub_off, n, nt, bhist, tile_cnt);
    const int64_t nb = (N + SB - 1) / SB;
    tl_block_sums<<<(int)nb, 256, 0, st>>>(nseg, N, bsums);
    count_launch(3);
    std::vector<unsigned long long> hs((size_t)nb);
    LM_CUDA(cudaMemcpyAsync(hs.data(), bsums, (size_t)nb * 8, cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    unsigned long long run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const unsigned long long x = hs[b];
        hs[b] = run;
        run += x;
    }
    *n_segments = (int64_t)run;
    LM_CHECK(run <= (unsigned long long)Lt.cap && run < (1ull << 32), LM_ERR_NOMEM,
             "tile binning needs %llu segments, capacity %lld", run, (long long)Lt.cap);
    LM_CUDA(cudaMemcpyAsync(bsums, hs.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, st));
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
        LM_CHECK(pos == base_k[k + 1], LM_ERR_CUDA, "tile counts of subset %d do not add up", k);
    }
    io[n] = (int)items.size();
    LM_CHECK((int64_t)items.size() <= Lt.max_items, LM_ERR_NOMEM, "tile work items exceed capacity");
    LM_CUDA(cudaMemcpyAsync(tile_off, ho.data(), ho.size() * 4, cudaMemcpyHostToDevice, st));
    if (!items.empty())
        LM_CUDA(cudaMemcpyAsync(A.items, items.data(), items.size() * sizeof(TileItem), cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(A.item_off, io.data(), io.size() * 4, cudaMemcpyHostToDevice, st));
    const size_t fsm = (size_t)nt * 8;
    if (fsm > 48 * 1024) {
        cudaFuncSetAttribute(tl_fill_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        cudaFuncSetAttribute(tl_fill_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
    }
    if (two_d) tl_fill_kernel<true><<<nbb, 256, fsm, st>>>(A, bb, bhist, tile_off, total);
    else tl_fill_kernel<false><<<nbb, 256, fsm, st>>>(A, bb, bhist, tile_off, total);
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
