// Listmode projection kernels: P^LM x (Eq. lmop), its adjoint, the fused
// per-subset data update of Alg. 2 (forward projection, closed-form dual
// step of Eq. proxD, back-projection of the dual change divided by mu), the
// dual initialisation of Eq. (yinit), and the sensitivity image P^T 1.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "lm_internal.h"

namespace lmh {

static thread_local std::string g_err;

void set_error(const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

void clear_error() { g_err.clear(); }

static std::atomic<int64_t> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n); }
int64_t launch_total() { return g_launches.load(); }

int num_sms()
{
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        n = v;
    });
    return n;
}

int check_grid(const lm_grid* g)
{
    LM_CHECK(g != nullptr, LM_ERR_INVALID_ARG, "grid is NULL");
    for (int d = 0; d < 3; ++d) {
        LM_CHECK(g->n[d] >= 1, LM_ERR_INVALID_ARG, "grid n[%d] = %d < 1", d, g->n[d]);
        LM_CHECK(g->h[d] > 0.0f && std::isfinite(g->h[d]), LM_ERR_INVALID_ARG, "grid h[%d] must be > 0", d);
        LM_CHECK(std::isfinite(g->origin[d]), LM_ERR_INVALID_ARG, "grid origin[%d] not finite", d);
    }
    LM_CHECK(nvox(g) < (int64_t(1) << 31), LM_ERR_INVALID_ARG, "grid has 2^31 or more voxels");
    return LM_OK;
}

int tv_ndim(const lm_grid* g)
{
    int nd = 0;
    for (int d = 0; d < 3; ++d) nd += g->n[d] > 1;
    return nd;
}

int make_geo(const lm_scanner* sc, const lm_grid* g, const lm_tof* tof, lmk::Geo& G, bool need_scanner)
{
    int rc = check_grid(g);
    if (rc) return rc;
    std::memset(&G, 0, sizeof(G));
    for (int d = 0; d < 3; ++d) {
        G.n[d] = g->n[d];
        G.h[d] = g->h[d];
        G.o[d] = g->origin[d];
    }
    G.V = (int)nvox(g);
    if (need_scanner) {
        LM_CHECK(sc != nullptr && sc->xtal_xyz != nullptr, LM_ERR_INVALID_ARG, "scanner or crystal table is NULL");
        LM_CHECK(sc->n_rings >= 1 && sc->n_xtal >= 2, LM_ERR_INVALID_ARG, "scanner needs n_rings >= 1, n_xtal >= 2");
        LM_CHECK((int64_t)sc->n_rings * sc->n_xtal < (int64_t(1) << 27), LM_ERR_INVALID_ARG,
                 "scanner has 2^27 or more crystals");
        G.xtal = sc->xtal_xyz;
        G.n_det = sc->n_rings * sc->n_xtal;
    }
    LM_CHECK(tof != nullptr, LM_ERR_INVALID_ARG, "tof is NULL");
    if (tof->n_bins > 0) {
        LM_CHECK(tof->n_bins % 2 == 1 && tof->n_bins <= 255, LM_ERR_INVALID_ARG, "n_bins must be odd and <= 255");
        LM_CHECK(tof->sigma_mm > 0.0f && tof->bin_mm > 0.0f && tof->n_sigma > 0.0f, LM_ERR_INVALID_ARG,
                 "TOF sigma, bin and n_sigma must be > 0");
        G.tof_on = 1;
        G.M = (tof->n_bins - 1) / 2;
        G.bin = tof->bin_mm;
        G.W = tof->n_sigma * tof->sigma_mm;
        G.inv_s = (float)(1.0 / (std::sqrt(2.0) * (double)tof->sigma_mm));
    } else {
        LM_CHECK(tof->n_bins == 0, LM_ERR_INVALID_ARG, "n_bins must be >= 0");
    }
    return LM_OK;
}

}  // namespace lmh

using namespace lmk;
using lmh::EvArgs;

namespace {

// Dual step of the prior (Alg. 2 line 15): w+ = beta prox_{R^*}((w + S Kx)/beta)
// = v / max(1, |v|/beta) with v = w + S_{n+1} Kx, per voxel.
__device__ void prior_dual(const EvArgs& A)
{
    const int wp = A.wpar[A.u];
    const float* __restrict__ wc = A.w_cur[wp];
    float* __restrict__ wn = A.w_nxt[wp];
    const float* __restrict__ x = A.px;
    const int nx = A.G.n[0], ny = A.G.n[1], nz = A.G.n[2];
    const int V = A.G.V;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t jj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; jj < V; jj += stride) {
        const int j = (int)jj;
        const int ix = j % nx;
        const int iy = (j / nx) % ny;
        const int iz = j / (nx * ny);
        const float x0 = x[j];
        int c = 0;
        float vx = 0.0f, vy = 0.0f, vz = 0.0f;
        int cx = -1, cy = -1, cz = -1;
        if (nx > 1) { cx = c++; vx = fmaf(A.s_prior, ix < nx - 1 ? x[j + 1] - x0 : 0.0f, wc[(int64_t)cx * V + j]); }
        if (ny > 1) { cy = c++; vy = fmaf(A.s_prior, iy < ny - 1 ? x[j + nx] - x0 : 0.0f, wc[(int64_t)cy * V + j]); }
        if (nz > 1) { cz = c++; vz = fmaf(A.s_prior, iz < nz - 1 ? x[j + nx * ny] - x0 : 0.0f, wc[(int64_t)cz * V + j]); }
        const float nrm = sqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
        const float den = A.beta > 0.0f ? fmaxf(1.0f, nrm / A.beta) : 0.0f;
        if (cx >= 0) wn[(int64_t)cx * V + j] = den > 0.0f ? vx / den : 0.0f;
        if (cy >= 0) wn[(int64_t)cy * V + j] = den > 0.0f ? vy / den : 0.0f;
        if (cz >= 0) wn[(int64_t)cz * V + j] = den > 0.0f ? vz / den : 0.0f;
    }
}

template <int MODE>
struct ModeTraits {
    static constexpr bool gather = MODE == lmh::EV_FWD || MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1 ||
                                   MODE == lmh::EV_YINIT || MODE == lmh::EV_YINIT_FX1;
    static constexpr bool back_float = MODE == lmh::EV_BACK || MODE == lmh::EV_DATA || MODE == lmh::EV_YINIT;
    static constexpr bool back_fx = MODE == lmh::EV_BACK_FX;
    static constexpr bool needs_y = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1;
    static constexpr bool needs_mu = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1 || MODE == lmh::EV_YINIT ||
                                     MODE == lmh::EV_YINIT_FX1;
    static constexpr bool needs_s = needs_mu;
    static constexpr bool needs_vin = MODE == lmh::EV_BACK || MODE == lmh::EV_BACK_FX || MODE == lmh::EV_ABSMAX;
    static constexpr bool traverse = MODE != lmh::EV_ABSMAX;
    static constexpr bool count = MODE == lmh::EV_COUNT;
    static constexpr bool prior_branch = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1;
};

constexpr int PCACHE = 3;  // cached passes of 32 samples (96 samples) per lane

template <int MODE, bool TWO_D>
__global__ void __launch_bounds__(256) ev_kernel(const EvArgs A)
{
    using T = ModeTraits<MODE>;
    int64_t eb = A.e_begin, ee = A.e_end;
    if (A.seq != nullptr) {
        const int sel = A.seq[A.u];
        if (sel >= A.n_subsets) {
            if (T::prior_branch) prior_dual(A);
            return;
        }
        eb = A.sub_off[sel];
        ee = A.sub_off[sel + 1];
    }
    const Geo& G = A.G;
    const int lane = threadIdx.x & 31;
    const int tofmode = G.tof_on ? TOF_BIN : TOF_NONE;
    const bool has_yf = A.x_yf != nullptr || A.acc_yf != nullptr || A.acci_yf != nullptr;
    const int CH = A.chunk;
    const int64_t count = ee - eb;
    const int64_t nchunks = count > 0 ? (count + CH - 1) / CH : 0;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t total_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int fx_E = 0;
    float fx_scale = 1.0f;
    if (T::back_fx) {
        const float vmax = __uint_as_float(*A.maxbits);
        fx_E = fx_exponent(vmax, (long long)count, A.stepmax);
        fx_scale = ldexpf(1.0f, fx_E);
    }
    float wmax = 0.0f;  // per-lane max for the FX1 / ABSMAX modes
    int64_t it = 0;
    for (;;) {
        int64_t c;
        if (A.queue != nullptr) {
            unsigned long long cc = 0;
            if (lane == 0) cc = atomicAdd(A.queue, 1ULL);
            c = (int64_t)__shfl_sync(FULL, cc, 0);
        } else {
            c = warp_global + it * total_warps;
            ++it;
        }
        if (c >= nchunks) break;
        const int64_t e0 = eb + c * CH;
        const int nev = (int)min((int64_t)CH, ee - e0);
        int md1 = -1, md2 = -1, mt = 0;
        float mc = 1.0f, ms = 0.0f, my = 0.0f, mv = 0.0f, mmu = 1.0f;
        if (lane < nev) {
            const int64_t e = e0 + lane;
            md1 = A.det1[e];
            md2 = A.det2[e];
            if (A.tof) mt = A.tof[e];
            if (A.corr) mc = A.corr[e];
            if (T::needs_s) ms = A.contam[e];
            if (T::needs_y) my = A.y[e];
            if (T::needs_mu) mmu = (float)A.mu[e];
            if (T::needs_vin) mv = A.vin[e];
        }
        if (MODE == lmh::EV_ABSMAX) {
            if (lane < nev) wmax = fmaxf(wmax, fabsf(mc * mv));
            continue;
        }
        float r_out = 0.0f, r_y = 0.0f;
        for (int j = 0; j < nev; ++j) {
            const int d1 = __shfl_sync(FULL, md1, j);
            const int d2 = __shfl_sync(FULL, md2, j);
            const int m = __shfl_sync(FULL, mt, j);
            const float cj = __shfl_sync(FULL, mc, j);
            Lor L;
            bool ok = d1 >= 0 && d1 < G.n_det && d2 >= 0 && d2 < G.n_det && d1 != d2 &&
                      (tofmode == TOF_NONE || (m >= -G.M && m <= G.M));
            ok = ok && lor_setup(G, d1, d2, m, tofmode, has_yf, L);
            if (!ok) {
                L.i0 = 0;
                L.cnt = 0;
                L.yf = 0;
                L.sA = L.sB = L.sk = 0;
            }
            const int npass = (L.cnt + 31) >> 5;
            const int iend = L.i0 + L.cnt;
            float acc = 0.0f, acc1 = 0.0f;
            Smp cs[PCACHE];
            if (T::gather) {
                const float* __restrict__ img = L.yf ? A.x_yf : A.x_std;
#pragma unroll
                for (int p = 0; p < PCACHE; ++p) {
                    cs[p].base = 0;
                    cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
                    if (p < npass) {
                        const int i = L.i0 + p * 32 + lane;
                        if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, cs[p])) {
                            acc += gather<TWO_D>(img, L, cs[p]);
                            acc1 += wsum<TWO_D>(cs[p]);
                        } else {
                            cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
                        }
                    }
                }
                for (int p = PCACHE; p < npass; ++p) {
                    const int i = L.i0 + p * 32 + lane;
                    Smp s;
                    if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, s)) {
                        acc += gather<TWO_D>(img, L, s);
                        acc1 += wsum<TWO_D>(s);
                    }
                }
                acc = warp_sum(acc);
                acc1 = warp_sum(acc1);
            }
            // per-event scalar step (all lanes hold the same values)
            float bval = 0.0f;  // value to back-project (before the weights)
            if (MODE == lmh::EV_FWD) {
                if (lane == j) r_out = cj * acc;
            } else if (MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1) {
                const float sj = __shfl_sync(FULL, ms, j);
                const float yj = __shfl_sync(FULL, my, j);
                const float muj = __shfl_sync(FULL, mmu, j);
                const float p1 = cj * acc1;                            // (P^LM 1)_e
                const float Se = p1 > 0.0f ? A.gamma_rho / p1 : 0.0f;  // S_k = gamma rho / P^LM_{N_k} 1
                const float a = fmaf(Se, fmaf(cj, acc, sj), yj);       // y + S (P^LM x + s)
                const float yp = prox_dstar(a, muj * Se);
                const float v = (yp - yj) / muj;
                if (lane == j) {
                    r_y = yp;
                    r_out = v;
                }
                if (MODE == lmh::EV_DATA) bval = cj * v;
                else wmax = fmaxf(wmax, fabsf(cj * v));
            } else if (MODE == lmh::EV_YINIT || MODE == lmh::EV_YINIT_FX1) {
                const float sj = __shfl_sync(FULL, ms, j);
                const float muj = __shfl_sync(FULL, mmu, j);
                const float u = fmaf(cj, acc, sj);
                const float yv = 1.0f - muj / u;          // Eq. (yinit) with d -> mu
                const float v = (yv - 1.0f) / muj;        // = -1/u
                if (lane == j) {
                    r_y = yv;
                    r_out = v;
                }
                if (MODE == lmh::EV_YINIT) bval = cj * v;
                else wmax = fmaxf(wmax, fabsf(cj * v));
            } else if (MODE == lmh::EV_BACK || MODE == lmh::EV_BACK_FX) {
                bval = cj * __shfl_sync(FULL, mv, j);
            }
            if (T::back_float && bval != 0.0f) {
                float* acc_img = L.yf ? A.acc_yf : A.acc_std;
                if (T::gather) {
#pragma unroll
                    for (int p = 0; p < PCACHE; ++p)
                        if (p < npass) scatter<TWO_D>(acc_img, L, cs[p], bval);
                    for (int p = PCACHE; p < npass; ++p) {
                        const int i = L.i0 + p * 32 + lane;
                        Smp s;
                        if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, s)) scatter<TWO_D>(acc_img, L, s, bval);
                    }
                } else {
                    for (int p = 0; p < npass; ++p) {
                        const int i = L.i0 + p * 32 + lane;
                        Smp s;
                        if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, s)) scatter<TWO_D>(acc_img, L, s, bval);
                    }
                }
            }
            if (T::count) {
                unsigned long long ns = 0, nt = 0;
                for (int p = 0; p < npass; ++p) {
                    const int i = L.i0 + p * 32 + lane;
                    Smp s;
                    if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, s)) {
                        ns += 1;
                        nt += (s.w0 != 0.0f) + (s.w1 != 0.0f) + (s.w2 != 0.0f) + (s.w3 != 0.0f);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ns += __shfl_xor_sync(FULL, ns, o);
                    nt += __shfl_xor_sync(FULL, nt, o);
                }
                if (lane == 0) {
                    atomicAdd(A.acci_std, ns);
                    atomicAdd(A.acci_std + 1, nt);
                }
            }
            if (T::back_fx && bval != 0.0f) {
                unsigned long long* acc_img = L.yf ? A.acci_yf : A.acci_std;
                const float v2 = bval * fx_scale;
                for (int p = 0; p < npass; ++p) {
                    const int i = L.i0 + p * 32 + lane;
                    Smp s;
                    if (i < iend && sample_at<TWO_D>(G, L, tofmode, i, s)) scatter_fx<TWO_D>(acc_img, L, s, v2);
                }
            }
        }
        if (lane < nev) {
            const int64_t e = e0 + lane;
            if (MODE == lmh::EV_FWD) A.out[e] = r_out;
            if (MODE == lmh::EV_DATA || MODE == lmh::EV_YINIT) A.y[e] = r_y;
            if (MODE == lmh::EV_DATA_FX1 || MODE == lmh::EV_YINIT_FX1) {
                A.y[e] = r_y;
                A.out[e] = r_out;
            }
        }
    }
    if (MODE == lmh::EV_DATA_FX1 || MODE == lmh::EV_YINIT_FX1 || MODE == lmh::EV_ABSMAX) {
        // non-negative floats order like their bit patterns
        float m = wmax;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
        if (lane == 0 && m > 0.0f) atomicMax(A.maxbits, __float_as_uint(m));
    }
    if (A.queue != nullptr) {
        // the last warp to finish resets the counters for the next launch
        __syncwarp();
        if (lane == 0) {
            const unsigned tw = (unsigned)total_warps;
            const unsigned d = atomicAdd(A.done, 1u);
            if (d == tw - 1) {
                *A.queue = 0ULL;
                *A.done = 0u;
            }
        }
    }
}

template <int MODE, bool TWO_D>
int launch_mode(const EvArgs& a, int grid, cudaStream_t st)
{
    ev_kernel<MODE, TWO_D><<<grid, 256, 0, st>>>(a);
    lmh::count_launch();
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

template <int MODE, bool TWO_D>
int occupancy_grid()
{
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ev_kernel<MODE, TWO_D>, 256, 0) != cudaSuccess || bps < 1)
        bps = 1;
    return bps * lmh::num_sms();
}

// Sensitivity image: every canonical LOR, TOF-summed sample weights.
template <bool TWO_D>
__global__ void __launch_bounds__(256) sens_kernel(const Geo G, const float* __restrict__ lf, float* acc_std,
                                                   float* acc_yf, int64_t n_lor, int n_xtal, int n_rings)
{
    const int lane = threadIdx.x & 31;
    const int64_t wg = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int tofmode = G.tof_on ? TOF_SUM : TOF_NONE;
    const int64_t B = (int64_t)n_xtal * ((n_xtal - 1) / 2);
    const int64_t nr2 = (int64_t)n_rings * n_rings;
    for (int64_t l = wg; l < n_lor; l += tw) {
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
        const int d1 = r1 * n_xtal + c1, d2 = r2 * n_xtal + c2;
        Lor L;
        if (!lor_setup(G, d1, d2, 0, tofmode, acc_yf != nullptr, L)) continue;
        const float val = lf ? lf[l] : 1.0f;
        if (val == 0.0f) continue;
        float* acc = L.yf ? acc_yf : acc_std;
        const int npass = (L.cnt + 31) >> 5;
        for (int p = 0; p < npass; ++p) {
            const int i = L.i0 + p * 32 + lane;
            Smp s;
            if (i < L.i0 + L.cnt && sample_at<TWO_D>(G, L, tofmode, i, s)) scatter<TWO_D>(acc, L, s, val);
        }
    }
}

}  // namespace

namespace lmh {

int launch_events(int mode, bool two_d, const EvArgs& a, int grid, cudaStream_t st)
{
#define LM_CASE(M)                                                                   \
    case M:                                                                          \
        return two_d ? launch_mode<M, true>(a, grid, st) : launch_mode<M, false>(a, grid, st);
    switch (mode) {
        LM_CASE(EV_FWD)
        LM_CASE(EV_BACK)
        LM_CASE(EV_BACK_FX)
        LM_CASE(EV_DATA)
        LM_CASE(EV_DATA_FX1)
        LM_CASE(EV_YINIT)
        LM_CASE(EV_YINIT_FX1)
        LM_CASE(EV_ABSMAX)
        LM_CASE(EV_COUNT)
        default:
            return LM_ERR_INVALID_ARG;
    }
#undef LM_CASE
}

int ev_grid(int mode, bool two_d)
{
#define LM_CASE(M) \
    case M:        \
        return two_d ? occupancy_grid<M, true>() : occupancy_grid<M, false>();
    switch (mode) {
        LM_CASE(EV_FWD)
        LM_CASE(EV_BACK)
        LM_CASE(EV_BACK_FX)
        LM_CASE(EV_DATA)
        LM_CASE(EV_DATA_FX1)
        LM_CASE(EV_YINIT)
        LM_CASE(EV_YINIT_FX1)
        LM_CASE(EV_ABSMAX)
        LM_CASE(EV_COUNT)
        default:
            return num_sms();
    }
#undef LM_CASE
}

static int check_events(const lm_events* ev, bool need_corr_contam)
{
    LM_CHECK(ev != nullptr, LM_ERR_INVALID_ARG, "events is NULL");
    LM_CHECK(ev->n >= 0, LM_ERR_INVALID_ARG, "negative event count");
    if (ev->n == 0) return LM_OK;
    LM_CHECK(ev->det1 && ev->det2, LM_ERR_INVALID_ARG, "event detector arrays are NULL");
    if (need_corr_contam) LM_CHECK(ev->contam != nullptr, LM_ERR_INVALID_ARG, "event contamination is NULL");
    return LM_OK;
}

static float step_max(const lm_grid* g)
{
    return 2.0f * std::fmax(g->h[0], std::fmax(g->h[1], g->h[2]));
}

}  // namespace lmh

using namespace lmh;

extern "C" {

const char* lm_last_error(void) { return g_err.c_str(); }

int lm_version(void) { return 100; }

int64_t lm_n_lor(const lm_scanner* sc)
{
    if (!sc || sc->n_xtal < 2 || sc->n_rings < 1) return 0;
    return (int64_t)sc->n_xtal * (sc->n_xtal - 1) / 2 * sc->n_rings * sc->n_rings;
}

size_t lm_fwd_workspace_bytes(const lm_grid* grid)
{
    if (check_grid(grid)) return 0;
    return align_up((size_t)nvox(grid) * 4);
}

int lm_fwd(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const float* x, const lm_events* ev,
           float* p, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    rc = check_events(ev, false);
    if (rc) return rc;
    if (ev->n == 0) return LM_OK;
    LM_CHECK(x != nullptr && p != nullptr, LM_ERR_INVALID_ARG, "x or p is NULL");
    LM_CHECK(tof->n_bins == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    cudaStream_t st = S(stream);
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = G;
    a.x_std = x;
    if (ws != nullptr && ws_bytes >= lm_fwd_workspace_bytes(grid) && grid->n[1] > 1) {
        launch_transpose_to_yf(grid, x, (float*)ws, st);
        a.x_yf = (const float*)ws;
    }
    a.det1 = ev->det1;
    a.det2 = ev->det2;
    a.tof = ev->tof;
    a.corr = ev->corr;
    a.out = p;
    a.e_begin = 0;
    a.e_end = ev->n;
    a.chunk = 32;
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;  // single-ring scanner in the image plane
    rc = launch_events(EV_FWD, two_d, a, ev_grid(EV_FWD, two_d), st);
    LM_CHECK(rc == LM_OK, rc, "forward projection launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return LM_OK;
}

size_t lm_back_workspace_bytes(const lm_grid* grid, int deterministic)
{
    if (check_grid(grid)) return 0;
    const size_t V = (size_t)nvox(grid);
    if (deterministic) return 2 * align_up(V * 8) + 256;
    return align_up(V * 4);
}

int lm_back(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev, const float* v,
            float* img, int deterministic, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    rc = check_events(ev, false);
    if (rc) return rc;
    if (ev->n == 0) return LM_OK;
    LM_CHECK(v != nullptr && img != nullptr, LM_ERR_INVALID_ARG, "v or img is NULL");
    LM_CHECK(tof->n_bins == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    const size_t need = lm_back_workspace_bytes(grid, deterministic);
    LM_CHECK(!deterministic || (ws != nullptr && ws_bytes >= need), LM_ERR_NOMEM,
             "deterministic back-projection needs %zu workspace bytes", need);
    cudaStream_t st = S(stream);
    const size_t V = (size_t)nvox(grid);
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;  // single-ring scanner in the image plane
    const bool use_yf = grid->n[1] > 1 && ws != nullptr && ws_bytes >= need;
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = G;
    a.det1 = ev->det1;
    a.det2 = ev->det2;
    a.tof = ev->tof;
    a.corr = ev->corr;
    a.vin = v;
    a.e_begin = 0;
    a.e_end = ev->n;
    a.chunk = 32;
    a.stepmax = step_max(grid);
    if (!deterministic) {
        a.acc_std = img;
        if (use_yf) {
            a.acc_yf = (float*)ws;
            LM_CUDA(cudaMemsetAsync(ws, 0, V * 4, st));
        }
        rc = launch_events(EV_BACK, two_d, a, ev_grid(EV_BACK, two_d), st);
        LM_CHECK(rc == LM_OK, rc, "back-projection launch failed");
        if (use_yf) launch_add_yf_to_std(grid, img, (float*)ws, st);
        return LM_OK;
    }
    char* w = (char*)ws;
    unsigned long long* a_std = (unsigned long long*)w;
    unsigned long long* a_yf = (unsigned long long*)(w + align_up(V * 8));
    unsigned* maxbits = (unsigned*)(w + 2 * align_up(V * 8));
    LM_CUDA(cudaMemsetAsync(ws, 0, need, st));
    a.maxbits = maxbits;
    rc = launch_events(EV_ABSMAX, two_d, a, ev_grid(EV_ABSMAX, two_d), st);
    LM_CHECK(rc == LM_OK, rc, "max reduction launch failed");
    a.acci_std = a_std;
    a.acci_yf = grid->n[1] > 1 ? a_yf : nullptr;
    rc = launch_events(EV_BACK_FX, two_d, a, ev_grid(EV_BACK_FX, two_d), st);
    LM_CHECK(rc == LM_OK, rc, "fixed-point back-projection launch failed");
    launch_fold_fixed(grid, img, a_std, grid->n[1] > 1 ? a_yf : nullptr, maxbits, (long long)ev->n, a.stepmax, st);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

size_t lm_sens_workspace_bytes(const lm_grid* grid)
{
    if (check_grid(grid)) return 0;
    return align_up((size_t)nvox(grid) * 4);
}

int lm_sens(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const float* lor_factor, float* sens,
            void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    LM_CHECK(sens != nullptr, LM_ERR_INVALID_ARG, "sens is NULL");
    cudaStream_t st = S(stream);
    const size_t V = (size_t)nvox(grid);
    LM_CUDA(cudaMemsetAsync(sens, 0, V * 4, st));
    float* yf = nullptr;
    if (ws != nullptr && ws_bytes >= lm_sens_workspace_bytes(grid) && grid->n[1] > 1) {
        yf = (float*)ws;
        LM_CUDA(cudaMemsetAsync(yf, 0, V * 4, st));
    }
    const int64_t nl = lm_n_lor(sc);
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;  // single-ring scanner in the image plane
    int bps = 0;
    if (two_d)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sens_kernel<true>, 256, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sens_kernel<false>, 256, 0);
    if (bps < 1) bps = 1;
    int64_t want = (nl + 7) / 8;  // 8 warps per block
    int grid_n = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)bps * num_sms() * 4);
    if (two_d)
        sens_kernel<true><<<grid_n, 256, 0, st>>>(G, lor_factor, sens, yf, nl, sc->n_xtal, sc->n_rings);
    else
        sens_kernel<false><<<grid_n, 256, 0, st>>>(G, lor_factor, sens, yf, nl, sc->n_xtal, sc->n_rings);
    LM_CUDA(cudaGetLastError());
    count_launch();
    if (yf) launch_add_yf_to_std(grid, sens, yf, st);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int64_t lm_kernel_launches(void) { return launch_total(); }

int lm_traversal_stats(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
                       void* ws, size_t ws_bytes, int64_t* n_samples, int64_t* n_touches, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    rc = check_events(ev, false);
    if (rc) return rc;
    LM_CHECK(n_samples && n_touches, LM_ERR_INVALID_ARG, "NULL output");
    LM_CHECK(ws != nullptr && ws_bytes >= 16, LM_ERR_NOMEM, "statistics need 16 workspace bytes");
    *n_samples = 0;
    *n_touches = 0;
    if (ev->n == 0) return LM_OK;
    cudaStream_t st = S(stream);
    unsigned long long* cnt = (unsigned long long*)ws;
    LM_CUDA(cudaMemsetAsync(cnt, 0, 16, st));
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = G;
    a.det1 = ev->det1;
    a.det2 = ev->det2;
    a.tof = ev->tof;
    a.e_begin = 0;
    a.e_end = ev->n;
    a.chunk = 32;
    a.acci_std = cnt;
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;
    rc = launch_events(EV_COUNT, two_d, a, ev_grid(EV_COUNT, two_d), st);
    unsigned long long h[2] = {0, 0};
    cudaMemcpyAsync(h, cnt, 16, cudaMemcpyDeviceToHost, st);
    LM_CUDA(cudaStreamSynchronize(st));
    LM_CHECK(rc == LM_OK, rc, "statistics launch failed");
    *n_samples = (int64_t)h[0];
    *n_touches = (int64_t)h[1];
    return LM_OK;
}

}  // extern "C"
