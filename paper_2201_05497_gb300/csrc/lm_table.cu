// Data update of Alg. 2 (forward projection of the subset's events, the
// closed-form dual step of Eq. (proxD), back-projection of the dual change
// divided by mu) from a stored traversal table.
//
// The direct event kernel (lm_project.cu) sets up every event's traversal
// from the crystal table on each visit, hands each event's parameters to
// its lane group by a dozen and a half warp shuffles and divides three times
// per event; most of its issue slots go to that per-event work, which only
// ~46 samples share.  This path
//  * computes each event's traversal (reading 1 of the projector: principal
//    axis, clipped plane range, affine secondary coordinates, TOF coordinate,
//    sample length), 1/(P^LM 1)_e and 1/mu_e once per state (trav_build),
//    so a data update reads 40 bytes of table per event;
//  * stages the selected events of a 32-event chunk in shared memory (one
//    64-byte record each), from where a lane group reads its event with four
//    broadcast loads instead of shuffles; the group's first lane writes y+;
//  * runs the subset's x-principal events and the others in two launches
//    (phases), so that one image layout and one accumulator layout are live
//    in L2 at a time (15 + 31 MB on a 200 x 200 x 96 grid).
// Per sample the arithmetic is the direct kernel's (positions, TOF table,
// bilinear weights, gathers, fused multiply-adds and atomics in the same
// order), so the forward projections agree with it bit for bit for the same
// lane-group width; S_e and (y+ - y)/mu use the stored reciprocals, which
// moves them by rounding only.  The back-projection goes into the same
// z-paired accumulators as the direct kernel's, so the image passes are
// shared.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "lm_internal.h"

using namespace lmk;

namespace lmh {

bool trav_capable(const lm_grid* g)
{
    if (g->n[2] < 2 || g->n[1] < 2) return false;
    for (int d = 0; d < 3; ++d)
        if (g->n[d] >= (1 << 15)) return false;
    return true;
}

TravLayout trav_layout(const lm_grid* g, int64_t N)
{
    (void)g;
    TravLayout L;
    std::memset(&L, 0, sizeof(L));
    const size_t n = (size_t)std::max<int64_t>(N, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(bytes);
        return o;
    };
    L.r0 = take(n * 16);
    L.r1 = take(n * 16);
    L.meta = take(n * 8);
    L.total = off + 256;
    return L;
}

}  // namespace lmh

namespace {

using lmh::TOF_TAB_N;

// Packed plane range and principal axis of a table entry: i0 (15 bits),
// cnt (15 bits, 0 = inert event), k (2 bits).
__host__ __device__ __forceinline__ unsigned pack_meta(int i0, int cnt, int k)
{
    return (unsigned)i0 | ((unsigned)cnt << 15) | ((unsigned)k << 30);
}

// One thread per event: the traversal of reading 1 (lor_setup, the direct
// kernel's own set-up), 1/(P^LM 1)_e with (P^LM 1)_e = c_e times the sum over
// the event's samples of the in-grid bilinear weights times TOF weight times
// sample length (0 where that sum is 0: S_e = 0, an inert event), and 1/mu_e.
__global__ void trav_build_kernel(const Geo G, const int32_t* __restrict__ det1, const int32_t* __restrict__ det2,
                                  const int16_t* __restrict__ tofb, const float* __restrict__ corr,
                                  const uint16_t* __restrict__ mu, int64_t N, const float* __restrict__ tab,
                                  float4* __restrict__ r0, float4* __restrict__ r1, int2* __restrict__ meta)
{
    __shared__ float s_tab[TOF_TAB_N + 1];
    for (int k = threadIdx.x; k <= TOF_TAB_N; k += blockDim.x) s_tab[k] = tab[k];
    __syncthreads();
    const float inv_dt = (float)TOF_TAB_N / (2.0f * G.W);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const int d1 = det1[e], d2 = det2[e], m = (int)tofb[e];
        bool ok = d1 >= 0 && d1 < G.n_det && d2 >= 0 && d2 < G.n_det && d1 != d2 && m >= -G.M && m <= G.M;
        Lor L;
        ok = ok && lor_setup(G, d1, d2, m, TOF_BIN, true, L);
        float4 a = make_float4(0.0f, 0.0f, 0.0f, 0.0f), b = a;
        unsigned mw = 0u;
        if (ok) {
            lmh::lor_strides(G, L.k, true, L);  // extents (and strides) of the secondary axes
            float acc1 = 0.0f;
            for (int i = L.i0; i < L.i0 + L.cnt; ++i) {
                Smp s;
                if (lmh::sample_tab<false>(G, L, s_tab, inv_dt, i, s)) acc1 += wsum<false>(s);
            }
            const float p1 = (corr ? corr[e] : 1.0f) * acc1;
            a = make_float4(L.ua0, L.sa, L.ub0, L.sb);
            b = make_float4(L.tau0, L.dtau, L.step, p1 > 0.0f ? 1.0f / p1 : 0.0f);
            mw = pack_meta(L.i0, L.cnt, L.k);
        }
        r0[e] = a;
        r1[e] = b;
        meta[e] = make_int2((int)mw, __float_as_int(1.0f / (float)mu[e]));
    }
}

// floor(v) for -2^22 <= v < 2^22 as an int and as a float, by one addition
// rounded towards -inf: adding 1.5 * 2^23 leaves a float whose unit in the
// last place is 1, so the rounded sum is 1.5 * 2^23 + floor(v) exactly.
// Same values as floorf and the conversion, on the full-rate adder.
__device__ __forceinline__ int floor_i(float v, float& fl)
{
    const float t = __fadd_rd(v, 12582912.0f);
    fl = t - 12582912.0f;
    return __float_as_int(t) - 0x4B400000;
}

// Sample at plane i (fi = i as a float) of a traversal: the direct kernel's
// sample_tab arithmetic with the TOF table read as (value, slope) pairs
// (slope = the same float difference the direct kernel forms) and floors on
// the adder.  Returns false for a sample without weight.
__device__ __forceinline__ bool sample_t(const Geo& G, const Lor& L, const float2* tab2, float inv_dt, int i,
                                         float fi, Smp& s)
{
    const float tau = fmaf(fi, L.dtau, L.tau0);
    if (fabsf(tau) > G.W) return false;
    const float uu = fminf(fmaxf((tau + G.W) * inv_dt, 0.0f), (float)TOF_TAB_N);
    float kf;
    const int kq = min(floor_i(uu, kf), TOF_TAB_N - 1);
    const float f = uu - fminf(kf, (float)(TOF_TAB_N - 1));
    const float2 t = tab2[kq];
    const float wt = L.step * fmaf(f, t.y, t.x);
    if (wt == 0.0f) return false;
    const float ua = fmaf(fi, L.sa, L.ua0);
    float fla;
    const int ia = floor_i(ua, fla);
    const float fa = ua - fla;
    const float wa0 = ((unsigned)ia < (unsigned)L.nA) ? (1.0f - fa) : 0.0f;
    const float wa1 = ((unsigned)(ia + 1) < (unsigned)L.nA) ? fa : 0.0f;
    const float ub = fmaf(fi, L.sb, L.ub0);
    float flb;
    const int ib = floor_i(ub, flb);
    const float fb = ub - flb;
    const float wb0 = ((unsigned)ib < (unsigned)L.nB) ? (1.0f - fb) : 0.0f;
    const float wb1 = ((unsigned)(ib + 1) < (unsigned)L.nB) ? fb : 0.0f;
    s.base = i * L.sk + ia * L.sA + ib * L.sB;
    const float wtA0 = wt * wa0, wtA1 = wt * wa1;
    s.w0 = wtA0 * wb0;
    s.w1 = wtA1 * wb0;
    s.w2 = wtA0 * wb1;
    s.w3 = wtA1 * wb1;
    return (s.w0 != 0.0f) || (s.w1 != 0.0f) || (s.w2 != 0.0f) || (s.w3 != 0.0f);
}

// One selected event of a chunk, staged in shared memory.
struct alignas(16) EvRec {
    float4 g0;     // ua0, sa, ub0, sb
    float4 g1;     // tau0, dtau, step, 1/(P^LM 1)_e
    float4 d;      // c_e, s_e, y_e, mu_e
    unsigned mw;   // packed plane range and principal axis
    int lane;      // the event's place in its chunk
    float inv_mu;  // 1/mu_e
    float pad;
};

// One chunk of 32 consecutive events [e0, e0 + nev) of a data update by the
// calling warp: phase 0 processes its x-principal events, phase 1 the
// others, phase -1 all of them.  The lanes load their event's table entry
// and fields coalesced, with the streaming cache policy (read once per
// update), and stage the selected events in shared memory by rank; groups of
// G lanes then take them in turn, lane s of a group on planes i0 + s,
// i0 + s + G, ... as in the direct kernel, keeping up to 64/G samples per lane
// in registers for the back-projection.  x_std / x_yf: the image the update
// gathers from.
template <int G>
__device__ __forceinline__ void table_chunk(const lmh::TabArgs& A, const float* __restrict__ x_std,
                                            const float* __restrict__ x_yf, int64_t e0, int nev, int phase,
                                            const float2* s_tab, float inv_dt, EvRec* rec)
{
    constexpr int NG = 32 / G;
    constexpr int PC = 64 / G;
    const Geo& Gm = A.G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int64_t e = e0 + lane;
    const bool in = lane < nev;
    const int2 mt = in ? __ldcs(A.meta + e) : make_int2(0, 0);
    const unsigned mw = (unsigned)mt.x;
    const int mk = (int)(mw >> 30);
    const bool mine = in && ((mw >> 15) & 0x7FFFu) != 0u && (phase < 0 || ((mk == 0) == (phase == 0)));
    const unsigned mask = __ballot_sync(FULL, mine);
    if (mask == 0u) return;
    if (mine) {
        EvRec& r = rec[__popc(mask & ((1u << lane) - 1u))];
        r.g0 = __ldcs(A.r0 + e);
        r.g1 = __ldcs(A.r1 + e);
        r.d = make_float4(A.corr ? __ldcs(A.corr + e) : 1.0f, __ldcs(A.contam + e), __ldcs(A.y + e),
                          (float)__ldcs(reinterpret_cast<const unsigned short*>(A.mu) + e));
        r.mw = mw;
        r.lane = lane;
        r.inv_mu = __int_as_float(mt.y);
    }
    __syncwarp();
    const int nm = __popc(mask);
    for (int b0 = 0; b0 < nm; b0 += NG) {
        const bool valid = b0 + grp < nm;
        const EvRec& R = rec[valid ? b0 + grp : b0];
        const float4 g0 = R.g0, g1 = R.g1, dd = R.d;
        const unsigned rw = R.mw;
        Lor E;
        E.i0 = (int)(rw & 0x7FFFu);
        E.cnt = valid ? (int)((rw >> 15) & 0x7FFFu) : 0;
        const int k = (int)(rw >> 30);
        E.ua0 = g0.x;
        E.sa = g0.y;
        E.ub0 = g0.z;
        E.sb = g0.w;
        E.tau0 = g1.x;
        E.dtau = g1.y;
        E.step = g1.z;
        lmh::lor_strides(Gm, k, true, E);
        E.k = k;
        const float* __restrict__ img = k == 1 ? x_yf : x_std;
        const int npass = (E.cnt + G - 1) / G;
        const int iend = E.i0 + E.cnt;
        const int ifirst = E.i0 + sub;
        const float ffirst = (float)ifirst;
        float acc = 0.0f;
        Smp cs[PC];
#pragma unroll
        for (int p = 0; p < PC; ++p) {
            cs[p].base = 0;
            cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
            if (p < npass) {
                const int i = ifirst + p * G;
                if (i < iend && sample_t(Gm, E, s_tab, inv_dt, i, ffirst + (float)(p * G), cs[p]))
                    acc += gather<false>(img, E, cs[p]);
                else
                    cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
            }
        }
        for (int p = PC; p < npass; ++p) {
            const int i = ifirst + p * G;
            Smp s;
            if (i < iend && sample_t(Gm, E, s_tab, inv_dt, i, (float)i, s)) acc += gather<false>(img, E, s);
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        // dual step of Eq. (proxD) with the listmode step mu_e S_e
        const float cj = dd.x, sj = dd.y, yj = dd.z, muj = dd.w;
        const float Se = A.gamma_rho * g1.w;                  // S_e = gamma rho / (P^LM 1)_e
        const float a = fmaf(Se, fmaf(cj, acc, sj), yj);      // y + S (P^LM x + s)
        const float yp = prox_dstar(a, muj * Se);
        const float v = (yp - yj) * R.inv_mu;                 // (y+ - y) / mu
        if (valid && sub == 0) __stcs(A.y + e0 + R.lane, yp);
        const float bval = valid ? cj * v : 0.0f;
        if (bval != 0.0f) {
            float* acc_img = k == 1 ? A.acc_yf : A.acc_std;
#pragma unroll
            for (int p = 0; p < PC; ++p)
                if (p < npass) scatter_pairs<false>(acc_img, E, cs[p], bval);
            for (int p = PC; p < npass; ++p) {
                const int i = ifirst + p * G;
                Smp s;
                if (i < iend && sample_t(Gm, E, s_tab, inv_dt, i, (float)i, s))
                    scatter_pairs<false>(acc_img, E, s, bval);
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void fill_tab2(float2* s_tab, const float* tab)
{
    for (int k = threadIdx.x; k < TOF_TAB_N; k += blockDim.x) {
        const float a = tab[k];
        s_tab[k] = make_float2(a, tab[k + 1] - a);
    }
}

// The self-resetting work counter: the last warp to finish clears it.
__device__ __forceinline__ void release_queue(unsigned long long* queue, unsigned* done)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        const unsigned tw = (unsigned)((gridDim.x * blockDim.x) >> 5);
        const unsigned d = atomicAdd(done, 1u);
        if (d == tw - 1) {
            *queue = 0ULL;
            *done = 0u;
        }
    }
}

// Data update of one subset from the traversal table: warps take the
// subset's chunks from a self-resetting counter (table_chunk).
template <int G, int MINB>
__global__ void __launch_bounds__(256, MINB) ev_table_kernel(const lmh::TabArgs A)
{
    __shared__ float2 s_tab[TOF_TAB_N];
    __shared__ EvRec s_rec[8][32];
    int64_t eb = A.e_begin, ee = A.e_end;
    if (A.seq != nullptr) {
        const int sel = A.seq[A.u];
        if (sel >= A.n_subsets) return;
        eb = A.sub_off[sel];
        ee = A.sub_off[sel + 1];
    }
    fill_tab2(s_tab, A.tof_tab);
    __syncthreads();
    const float inv_dt = (float)TOF_TAB_N / (2.0f * A.G.W);
    const int lane = threadIdx.x & 31;
    const int64_t count = ee - eb;
    const int64_t nch = count > 0 ? (count + 31) / 32 : 0;
    EvRec* rec = s_rec[threadIdx.x >> 5];
    for (;;) {
        unsigned long long cc = 0;
        if (lane == 0) cc = atomicAdd(A.queue, 1ULL);
        const int64_t c = (int64_t)__shfl_sync(FULL, cc, 0);
        if (c >= nch) break;
        const int64_t e0 = eb + c * 32;
        table_chunk<G>(A, A.x_std, A.x_yf, e0, (int)min((int64_t)32, ee - e0), A.phase, s_tab, inv_dt, rec);
    }
    release_queue(A.queue, A.done);
}

// The data updates of every active frame of a batch at update u, from their
// traversal tables: the work items are the 32-event chunks of each frame's
// selected subset (frames at a prior update have none: their dual step runs
// in the image pass), found through a prefix table in shared memory.
template <int G, int MINB>
__global__ void __launch_bounds__(256, MINB) ev_table_batch_kernel(const lmh::BatchTabArgs B)
{
    extern __shared__ float2 s_tab[];  // TOF_TAB_N pairs (dynamic: with the tables below above 48 KB)
    __shared__ EvRec s_rec[8][32];
    __shared__ long long s_pre[lmh::BATCH_MAX + 1];
    __shared__ long long s_eb[lmh::BATCH_MAX];
    __shared__ long long s_ee[lmh::BATCH_MAX];
    const int cap = B.cap;
    const int par = B.u & 1;
    if (threadIdx.x < cap) {
        const int s = threadIdx.x;
        long long items = 0, eb = 0, ee = 0;
        if (B.active[s]) {
            const lmh::TabArgs& A = B.slots[s];
            const int sel = B.seqs[(size_t)s * B.seq_stride + B.u];
            if (sel < A.n_subsets) {
                eb = A.sub_off[sel];
                ee = A.sub_off[sel + 1];
                items = (ee - eb + 31) / 32;
            }
        }
        s_eb[threadIdx.x] = eb;
        s_ee[threadIdx.x] = ee;
        s_pre[threadIdx.x + 1] = items;
    }
    fill_tab2(s_tab, B.tof_tab);
    __syncthreads();
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int s = 0; s < cap; ++s) s_pre[s + 1] += s_pre[s];
    }
    __syncthreads();
    const long long total = s_pre[cap];
    const float inv_dt = (float)TOF_TAB_N / (2.0f * B.tof_W);
    const int lane = threadIdx.x & 31;
    EvRec* rec = s_rec[threadIdx.x >> 5];
    for (;;) {
        unsigned long long cc = 0;
        if (lane == 0) cc = atomicAdd(B.queue, 1ULL);
        const long long c = (long long)__shfl_sync(FULL, cc, 0);
        if (c >= total) break;
        int s = 0;
        while (s_pre[s + 1] <= c) ++s;
        const lmh::TabArgs& A = B.slots[s];
        const int64_t e0 = s_eb[s] + (c - s_pre[s]) * 32;
        table_chunk<G>(A, A.xs[par], A.xyfs[par], e0, (int)min((long long)32, s_ee[s] - e0), -1, s_tab, inv_dt, rec);
    }
    release_queue(B.queue, B.done);
}

}  // namespace

namespace lmh {

int trav_build(const Geo& G, const lm_events& ev, const uint16_t* mu, const float* tof_tab, const TravLayout& L,
               char* base, cudaStream_t st)
{
    LM_CHECK(G.tof_on && tof_tab != nullptr, LM_ERR_INVALID_ARG, "the traversal table needs TOF data");
    if (ev.n <= 0) return LM_OK;
    const int grid = std::max<int64_t>(1, std::min<int64_t>((ev.n + 255) / 256, (int64_t)num_sms() * 8));
    trav_build_kernel<<<grid, 256, 0, st>>>(G, ev.det1, ev.det2, ev.tof, ev.corr, mu, ev.n, tof_tab,
                                            (float4*)(base + L.r0), (float4*)(base + L.r1), (int2*)(base + L.meta));
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// Lane-group widths and the resident blocks each variant is compiled for
// (registers per thread): width 32 with 3 or 4 blocks per SM, 16 and 8 with 2.
template <int G, int MINB>
static int table_blocks()
{
    static int nb = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ev_table_kernel<G, MINB>, 256, 0) != cudaSuccess ||
            b < 1)
            b = 1;
        nb = b;
    });
    return nb;
}

int table_grid(int variant)
{
    int b = 1;
    switch (variant) {
    case 8: b = table_blocks<8, 2>(); break;
    case 16: b = table_blocks<16, 2>(); break;
    case 32: b = table_blocks<32, 3>(); break;
    case 33: b = table_blocks<32, 4>(); break;
    default: break;
    }
    return num_sms() * b;
}

template <int G, int MINB>
static void batch_attr()
{
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(ev_table_batch_kernel<G, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(TOF_TAB_N * sizeof(float2)));
    });
}

int launch_table_batch(const BatchTabArgs& b, int variant, int grid, cudaStream_t st)
{
    const size_t dyn = TOF_TAB_N * sizeof(float2);
    switch (variant) {
    case 8: batch_attr<8, 2>(); ev_table_batch_kernel<8, 2><<<grid, 256, dyn, st>>>(b); break;
    case 16: batch_attr<16, 2>(); ev_table_batch_kernel<16, 2><<<grid, 256, dyn, st>>>(b); break;
    case 32: batch_attr<32, 3>(); ev_table_batch_kernel<32, 3><<<grid, 256, dyn, st>>>(b); break;
    case 33: batch_attr<32, 4>(); ev_table_batch_kernel<32, 4><<<grid, 256, dyn, st>>>(b); break;
    default: set_error("unknown traversal-table kernel variant %d", variant); return LM_ERR_INVALID_ARG;
    }
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int launch_table_update(const TabArgs& a, int variant, int grid, cudaStream_t st)
{
    switch (variant) {
    case 8: ev_table_kernel<8, 2><<<grid, 256, 0, st>>>(a); break;
    case 16: ev_table_kernel<16, 2><<<grid, 256, 0, st>>>(a); break;
    case 32: ev_table_kernel<32, 3><<<grid, 256, 0, st>>>(a); break;
    case 33: ev_table_kernel<32, 4><<<grid, 256, 0, st>>>(a); break;
    default: set_error("unknown traversal-table kernel variant %d", variant); return LM_ERR_INVALID_ARG;
    }
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

}  // namespace lmh
