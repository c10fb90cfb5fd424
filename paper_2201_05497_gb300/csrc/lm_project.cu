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

void tof_table(const lm_tof* tof, float* tab)
{
    const double sig = tof->sigma_mm, D = tof->bin_mm, W = (double)tof->n_sigma * sig;
    const double s = std::sqrt(2.0) * sig;
    for (int k = 0; k <= TOF_TAB_N; ++k) {
        const double tau = -W + 2.0 * W * k / TOF_TAB_N;
        tab[k] = (float)(0.5 * (std::erf((tau + 0.5 * D) / s) - std::erf((tau - 0.5 * D) / s)));
    }
}

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

// Dual step of the prior at voxel j (prior update of Alg. 2):
// w+ = v / max(1, |v|/beta), v = w + S_{n+1} K x; K x is the forward
// difference vector, or (directional TV, A.xi set) its part perpendicular to
// the structural field.
__device__ __forceinline__ void prior_voxel(const EvArgs& A, const float* __restrict__ x,
                                            const float* __restrict__ wc, float* __restrict__ wn, int j)
{
    const int nx = A.G.n[0], ny = A.G.n[1], nz = A.G.n[2];
    const int V = A.G.V;
    const int ix = j % nx;
    const int iy = (j / nx) % ny;
    const int iz = j / (nx * ny);
    const float x0 = x[j];
    int c = 0;
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
    int cx = -1, cy = -1, cz = -1;
    if (nx > 1) { cx = c++; gx = ix < nx - 1 ? x[j + 1] - x0 : 0.0f; }
    if (ny > 1) { cy = c++; gy = iy < ny - 1 ? x[j + nx] - x0 : 0.0f; }
    if (nz > 1) { cz = c++; gz = iz < nz - 1 ? x[j + nx * ny] - x0 : 0.0f; }
    if (A.xi != nullptr) {
        const float* f = A.xi;
        dtv_perp(cx >= 0 ? f[(int64_t)cx * V + j] : 0.0f, cy >= 0 ? f[(int64_t)cy * V + j] : 0.0f,
                 cz >= 0 ? f[(int64_t)cz * V + j] : 0.0f, gx, gy, gz);
    }
    float vx = 0.0f, vy = 0.0f, vz = 0.0f;
    if (cx >= 0) vx = fmaf(A.s_prior, gx, wc[(int64_t)cx * V + j]);
    if (cy >= 0) vy = fmaf(A.s_prior, gy, wc[(int64_t)cy * V + j]);
    if (cz >= 0) vz = fmaf(A.s_prior, gz, wc[(int64_t)cz * V + j]);
    const float sc = tv_ball_scale(fmaf(vx, vx, fmaf(vy, vy, vz * vz)), A.beta);
    const float ox = __fmul_rn(vx, sc), oy = __fmul_rn(vy, sc), oz = __fmul_rn(vz, sc);
    if (cx >= 0) wn[(int64_t)cx * V + j] = ox;
    if (cy >= 0) wn[(int64_t)cy * V + j] = oy;
    if (cz >= 0) wn[(int64_t)cz * V + j] = oz;
    if (A.dtv_d != nullptr) {
        // P (w+ - w) for the image pass's K^T (w+ - w) = grad^T P (w+ - w)
        const float* f = A.xi;
        float dx = cx >= 0 ? ox - wc[(int64_t)cx * V + j] : 0.0f;
        float dy = cy >= 0 ? oy - wc[(int64_t)cy * V + j] : 0.0f;
        float dz = cz >= 0 ? oz - wc[(int64_t)cz * V + j] : 0.0f;
        dtv_perp(cx >= 0 ? f[(int64_t)cx * V + j] : 0.0f, cy >= 0 ? f[(int64_t)cy * V + j] : 0.0f,
                 cz >= 0 ? f[(int64_t)cz * V + j] : 0.0f, dx, dy, dz);
        if (cx >= 0) A.dtv_d[(int64_t)cx * V + j] = dx;
        if (cy >= 0) A.dtv_d[(int64_t)cy * V + j] = dy;
        if (cz >= 0) A.dtv_d[(int64_t)cz * V + j] = dz;
    }
}

__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float f4(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }

// The prior's dual step at the four voxels j..j+3 of one image row (nx a
// multiple of 4, so the quad never crosses a row and every 16-byte access is
// aligned): all loads are issued before any arithmetic.  Same arithmetic per
// voxel as prior_voxel.
__device__ __forceinline__ void prior_quad(const EvArgs& A, const float* __restrict__ x,
                                           const float* __restrict__ wc, float* __restrict__ wn, int64_t j)
{
    const int nx = A.G.n[0], ny = A.G.n[1], nz = A.G.n[2];
    const int64_t V = A.G.V;
    const int ix = (int)(j % nx);
    const int64_t r = j / nx;
    const int iy = (int)(r % ny);
    const int iz = (int)(r / ny);
    const bool hx = nx > 1, hy = ny > 1, hz = nz > 1;
    const int cy = hx ? 1 : 0, cz = cy + (hy ? 1 : 0);
    const bool iny = iy < ny - 1, inz = iz < nz - 1;
    const float4 xc = ld4(x + j);
    const float xr = (hx && ix + 4 < nx) ? __ldg(x + j + 4) : 0.0f;
    const float4 xy = (hy && iny) ? ld4(x + j + nx) : xc;
    const float4 xz = (hz && inz) ? ld4(x + j + (int64_t)nx * ny) : xc;
    const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 wx = hx ? ld4(wc + j) : z4;
    const float4 wy = hy ? ld4(wc + (int64_t)cy * V + j) : z4;
    const float4 wz = hz ? ld4(wc + (int64_t)cz * V + j) : z4;
    const bool dtv = A.xi != nullptr;
    const float4 fx = (dtv && hx) ? ld4(A.xi + j) : z4;
    const float4 fy = (dtv && hy) ? ld4(A.xi + (int64_t)cy * V + j) : z4;
    const float4 fz = (dtv && hz) ? ld4(A.xi + (int64_t)cz * V + j) : z4;
    float ox[4], oy[4], oz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float x0 = f4(xc, k);
        const float xn = k < 3 ? f4(xc, k + 1) : xr;
        float gx = hx ? (ix + k < nx - 1 ? xn - x0 : 0.0f) : 0.0f;
        float gy = hy ? (iny ? f4(xy, k) - x0 : 0.0f) : 0.0f;
        float gz = hz ? (inz ? f4(xz, k) - x0 : 0.0f) : 0.0f;
        if (dtv) dtv_perp(f4(fx, k), f4(fy, k), f4(fz, k), gx, gy, gz);
        const float vx = hx ? fmaf(A.s_prior, gx, f4(wx, k)) : 0.0f;
        const float vy = hy ? fmaf(A.s_prior, gy, f4(wy, k)) : 0.0f;
        const float vz = hz ? fmaf(A.s_prior, gz, f4(wz, k)) : 0.0f;
        const float sc = tv_ball_scale(fmaf(vx, vx, fmaf(vy, vy, vz * vz)), A.beta);
        ox[k] = __fmul_rn(vx, sc);
        oy[k] = __fmul_rn(vy, sc);
        oz[k] = __fmul_rn(vz, sc);
    }
    if (dtv && A.dtv_d != nullptr) {
        // P (w+ - w) for the image pass's K^T (w+ - w) = grad^T P (w+ - w)
        float dx[4], dy[4], dz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dx[k] = hx ? ox[k] - f4(wx, k) : 0.0f;
            dy[k] = hy ? oy[k] - f4(wy, k) : 0.0f;
            dz[k] = hz ? oz[k] - f4(wz, k) : 0.0f;
            dtv_perp(f4(fx, k), f4(fy, k), f4(fz, k), dx[k], dy[k], dz[k]);
        }
        float* D = A.dtv_d;
        if (hx) *reinterpret_cast<float4*>(D + j) = make_float4(dx[0], dx[1], dx[2], dx[3]);
        if (hy) *reinterpret_cast<float4*>(D + (int64_t)cy * V + j) = make_float4(dy[0], dy[1], dy[2], dy[3]);
        if (hz) *reinterpret_cast<float4*>(D + (int64_t)cz * V + j) = make_float4(dz[0], dz[1], dz[2], dz[3]);
    }
    if (hx) *reinterpret_cast<float4*>(wn + j) = make_float4(ox[0], ox[1], ox[2], ox[3]);
    if (hy) *reinterpret_cast<float4*>(wn + (int64_t)cy * V + j) = make_float4(oy[0], oy[1], oy[2], oy[3]);
    if (hz) *reinterpret_cast<float4*>(wn + (int64_t)cz * V + j) = make_float4(oz[0], oz[1], oz[2], oz[3]);
}

// Prior dual step over voxels [j0, j1) by `nthr` threads numbered t: quads
// when rows are a multiple of 4 long, single voxels otherwise.
__device__ __forceinline__ void prior_range(const EvArgs& A, const float* __restrict__ x, int wp, int64_t j0,
                                            int64_t j1, int64_t t, int64_t nthr)
{
    const float* wc = A.w_cur[wp];
    float* wn = A.w_nxt[wp];
    if ((A.G.n[0] & 3) == 0) {
        for (int64_t j = j0 + 4 * t; j < j1; j += 4 * nthr) prior_quad(A, x, wc, wn, j);
    } else {
        for (int64_t j = j0 + t; j < j1; j += nthr) prior_voxel(A, x, wc, wn, (int)j);
    }
}

// The prior's dual step over the whole image, grid-stride.
__device__ __noinline__ void prior_dual(const EvArgs& A)
{
    prior_range(A, A.px, A.wpar[A.u], 0, A.G.V, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                (int64_t)gridDim.x * blockDim.x);
}

// Sinogram bin e of the generated layout (lm_params.sinogram = 2): the subset
// holding e (binary search of the offsets), then the bin's transaxial pair,
// ring pair and TOF bin in the order lm_sino_setup writes them: pairs in
// their subset's list, ring pairs, TOF bins; canonical detectors.
__device__ __forceinline__ void gen_bin(const EvArgs& A, int64_t e, int& d1, int& d2, int& m, float& c)
{
    int lo = 0, hi = A.n_subsets;  // sub_off[lo] <= e < sub_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (A.sub_off[mid] <= e) lo = mid;
        else hi = mid;
    }
    const int nr = A.g_rings, nb = A.g_nb, nx = A.g_xtal;
    const int64_t nr2 = (int64_t)nr * nr;
    const int64_t per_q = nr2 * nb;
    const int64_t pos = e - A.sub_off[lo];
    const int64_t qr = pos / per_q;
    const int64_t rem = pos - qr * per_q;
    const int rr = (int)(rem / nb);
    const int mi = (int)(rem - (int64_t)rr * nb);
    const int64_t qq = A.g_q[A.g_qoff[lo] + qr];
    const int64_t B = (int64_t)nx * ((nx - 1) / 2);
    int c1, c2;
    if (qq < B) {
        c1 = (int)(qq % nx);
        c2 = (int)((c1 + 1 + qq / nx) % nx);
    } else {
        c1 = (int)(qq - B);
        c2 = c1 + nx / 2;
    }
    const int r1 = rr / nr, r2 = rr - r1 * nr;
    d1 = r1 * nx + c1;
    d2 = r2 * nx + c2;
    m = mi - (nb - 1) / 2;
    c = A.g_lorf ? A.g_lorf[qq * nr2 + rr] : 1.0f;
}

template <int MODE>
struct ModeTraits {
    static constexpr bool gather = MODE == lmh::EV_FWD || MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1 ||
                                   MODE == lmh::EV_YINIT || MODE == lmh::EV_YINIT_FX1 || MODE == lmh::EV_EM;
    static constexpr bool back_float =
        MODE == lmh::EV_BACK || MODE == lmh::EV_DATA || MODE == lmh::EV_YINIT || MODE == lmh::EV_EM;
    static constexpr bool back_fx = MODE == lmh::EV_BACK_FX;
    static constexpr bool needs_y = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1;
    static constexpr bool needs_mu = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1 || MODE == lmh::EV_YINIT ||
                                     MODE == lmh::EV_YINIT_FX1;
    static constexpr bool needs_s = needs_mu || MODE == lmh::EV_EM;
    static constexpr bool needs_vin = MODE == lmh::EV_BACK || MODE == lmh::EV_BACK_FX || MODE == lmh::EV_ABSMAX;
    static constexpr bool traverse = MODE != lmh::EV_ABSMAX;
    static constexpr bool count = MODE == lmh::EV_COUNT;
    static constexpr bool prior_branch = MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1;
};

// Cached sample capacity per lane (3D: the 3-sigma window spans at most ~62
// planes of 2.5 mm; 2D: ~80 planes of 2 mm); larger traversals recompute.
template <bool TWO_D, int G>
struct Cache {
    static constexpr int passes = ((TWO_D ? 80 : 64) + G - 1) / G;
};

using lmh::sample_tab;
using lmh::tof_weight_tab;

// One sample, TOF weight from the table when the caller gave one.
template <bool TWO_D>
__device__ __forceinline__ bool sample_any(const Geo& G, const Lor& L, int tofmode, const float* tab, float inv_dt,
                                           int i, Smp& s)
{
    if (tofmode == TOF_BIN && tab != nullptr) return sample_tab<TWO_D>(G, L, tab, inv_dt, i, s);
    return sample_at<TWO_D>(G, L, tofmode, i, s);
}

using lmh::lor_strides;

// One chunk of events [e0, e0 + nev) processed by the calling warp (see
// ev_kernel).  x_std_in / x_yf_in: the image being projected, both layouts.
template <int MODE, bool TWO_D, int G>
__device__ __forceinline__ void event_chunk(const EvArgs& A, const float* __restrict__ x_std_in,
                                            const float* __restrict__ x_yf_in, bool has_yf, int64_t e0, int nev,
                                            const float* tab, float inv_dt, float fx_scale, float& wmax,
                                            unsigned long long& cnt_s, unsigned long long& cnt_t)
{
    using T = ModeTraits<MODE>;
    constexpr int NG = 32 / G;
    constexpr int PC = Cache<TWO_D, G>::passes;
    const Geo& Gm = A.G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int tofmode = Gm.tof_on ? TOF_BIN : TOF_NONE;
    const int R = (nev + NG - 1) / NG;  // rounds; event (grp*R + r) is owned by lane grp*G + r
    const int q = grp * R + sub;
    const bool own = sub < R && q < nev;
    // ---- per-lane load and set-up of the owned event ----
    float mc = 1.0f, ms = 0.0f, my = 0.0f, mv = 0.0f, mmu = 1.0f;
    Lor L;
    int mk = 0;
    bool mok = false;
    if (own) {
        const int64_t e = e0 + q;
        int d1, d2, m;
        if (A.sino == 2) {
            gen_bin(A, e, d1, d2, m, mc);
            ms = A.g_s;
        } else {
            d1 = A.det1[e];
            d2 = A.det2[e];
            m = A.tof ? (int)A.tof[e] : 0;
            if (A.corr) mc = A.corr[e];
            if (T::needs_s) ms = A.contam[e];
        }
        if (T::needs_y) my = A.y[e];
        if (T::needs_mu) mmu = (float)A.mu[e];
        if (T::needs_vin) mv = A.vin[e];
        if (T::traverse) {
            mok = d1 >= 0 && d1 < Gm.n_det && d2 >= 0 && d2 < Gm.n_det && d1 != d2 &&
                  (tofmode == TOF_NONE || (m >= -Gm.M && m <= Gm.M));
            mok = mok && lor_setup(Gm, d1, d2, m, tofmode, has_yf, L);
            if (mok) mk = L.k;
        }
    }
    if (MODE == lmh::EV_ABSMAX) {
        if (own) wmax = fmaxf(wmax, fabsf(mc * mv));
        return;
    }
    if (!mok) {
        L.i0 = 0;
        L.cnt = 0;
        L.ua0 = L.sa = L.ub0 = L.sb = L.tau0 = L.dtau = L.step = 0.0f;
    }
    float r_out = 0.0f, r_y = 0.0f;
    for (int r = 0; r < R; ++r) {
        const int src = grp * G + r;
        // parameters of this group's event from its owner lane
        Lor E;
        E.i0 = __shfl_sync(FULL, L.i0, src);
        E.cnt = __shfl_sync(FULL, L.cnt, src);
        const int k = __shfl_sync(FULL, mk, src);
        E.ua0 = __shfl_sync(FULL, L.ua0, src);
        E.sa = __shfl_sync(FULL, L.sa, src);
        if (!TWO_D) {
            E.ub0 = __shfl_sync(FULL, L.ub0, src);
            E.sb = __shfl_sync(FULL, L.sb, src);
        } else {
            E.ub0 = 0.0f;
            E.sb = 0.0f;
        }
        E.tau0 = __shfl_sync(FULL, L.tau0, src);
        E.dtau = __shfl_sync(FULL, L.dtau, src);
        E.step = __shfl_sync(FULL, L.step, src);
        const float cj = __shfl_sync(FULL, mc, src);
        const bool valid = r < R && (grp * R + r) < nev;
        if (!valid) E.cnt = 0;
        lor_strides(Gm, k, has_yf, E);
        E.k = k;
        const int npass = (E.cnt + G - 1) / G;
        const int iend = E.i0 + E.cnt;
        float acc = 0.0f, acc1 = 0.0f;
        Smp cs[PC];
        if (T::gather) {
            const float* __restrict__ img = E.yf ? x_yf_in : x_std_in;
#pragma unroll
            for (int p = 0; p < PC; ++p) {
                cs[p].base = 0;
                cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
                if (p < npass) {
                    const int i = E.i0 + p * G + sub;
                    if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, cs[p])) {
                        acc += gather<TWO_D>(img, E, cs[p]);
                        acc1 += wsum<TWO_D>(cs[p]);
                    } else {
                        cs[p].w0 = cs[p].w1 = cs[p].w2 = cs[p].w3 = 0.0f;
                    }
                }
            }
            for (int p = PC; p < npass; ++p) {
                const int i = E.i0 + p * G + sub;
                Smp s;
                if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, s)) {
                    acc += gather<TWO_D>(img, E, s);
                    acc1 += wsum<TWO_D>(s);
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(FULL, acc, o);
                acc1 += __shfl_xor_sync(FULL, acc1, o);
            }
        }
        float bval = 0.0f;
        if (MODE == lmh::EV_FWD) {
            if (lane == src) r_out = cj * acc;
        } else if (MODE == lmh::EV_DATA || MODE == lmh::EV_DATA_FX1) {
            const float sj = __shfl_sync(FULL, ms, src);
            const float yj = __shfl_sync(FULL, my, src);
            const float muj = __shfl_sync(FULL, mmu, src);
            const float p1 = cj * acc1;                            // (P^LM 1)_e
            const float Se = p1 > 0.0f ? A.gamma_rho / p1 : 0.0f;  // S_k = gamma rho / P^LM_{N_k} 1
            const float a = fmaf(Se, fmaf(cj, acc, sj), yj);       // y + S (P^LM x + s)
            const float yp = prox_dstar(a, muj * Se);
            // Alg. 2 back-projects (y+ - y)/mu; Alg. 1 on sinogram bins (mu = d_b) y+ - y
            const float v = A.sino ? yp - yj : (yp - yj) / muj;
            if (lane == src) {
                r_y = yp;
                r_out = v;
            }
            if (MODE == lmh::EV_DATA) bval = valid ? cj * v : 0.0f;
            else if (valid) wmax = fmaxf(wmax, fabsf(cj * v));
        } else if (MODE == lmh::EV_YINIT || MODE == lmh::EV_YINIT_FX1) {
            const float sj = __shfl_sync(FULL, ms, src);
            const float muj = __shfl_sync(FULL, mmu, src);
            const float u = fmaf(cj, acc, sj);
            const float yv = 1.0f - muj / u;                       // Eq. (yinit) with d -> mu
            const float v = A.sino ? yv - 1.0f : (yv - 1.0f) / muj;  // listmode: -1/u
            if (lane == src) {
                r_y = yv;
                r_out = v;
            }
            if (MODE == lmh::EV_YINIT) bval = valid ? cj * v : 0.0f;
            else if (valid) wmax = fmaxf(wmax, fabsf(cj * v));
        } else if (MODE == lmh::EV_EM) {
            // subset EM step of Alg. 3: back-project c_e / (c_e J_e x + s_e)
            const float sj = __shfl_sync(FULL, ms, src);
            const float u = fmaf(cj, acc, sj);
            bval = (valid && u > 0.0f) ? cj / u : 0.0f;
        } else if (MODE == lmh::EV_BACK || MODE == lmh::EV_BACK_FX) {
            // every lane takes part in the shuffle; groups without an event discard the value
            const float vj = __shfl_sync(FULL, mv, src);
            bval = valid ? cj * vj : 0.0f;
        }
        if (T::back_float && bval != 0.0f) {
            float* acc_img = E.yf ? A.acc_yf : A.acc_std;
            auto put = [&](const Smp& s) {
                if (A.acc_pairs) scatter_pairs<TWO_D>(acc_img, E, s, bval);
                else scatter<TWO_D>(acc_img, E, s, bval);
            };
            if (T::gather) {
#pragma unroll
                for (int p = 0; p < PC; ++p)
                    if (p < npass) put(cs[p]);
                for (int p = PC; p < npass; ++p) {
                    const int i = E.i0 + p * G + sub;
                    Smp s;
                    if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, s)) put(s);
                }
            } else {
                for (int p = 0; p < npass; ++p) {
                    const int i = E.i0 + p * G + sub;
                    Smp s;
                    if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, s)) put(s);
                }
            }
        }
        if (T::count) {
            for (int p = 0; p < npass; ++p) {
                const int i = E.i0 + p * G + sub;
                Smp s;
                if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, s)) {
                    cnt_s += 1;
                    cnt_t += (s.w0 != 0.0f) + (s.w1 != 0.0f) + (s.w2 != 0.0f) + (s.w3 != 0.0f);
                }
            }
        }
        if (T::back_fx && bval != 0.0f) {
            unsigned long long* acc_img = E.yf ? A.acci_yf : A.acci_std;
            const float v2 = bval * fx_scale;
            for (int p = 0; p < npass; ++p) {
                const int i = E.i0 + p * G + sub;
                Smp s;
                if (i < iend && sample_any<TWO_D>(Gm, E, tofmode, tab, inv_dt, i, s))
                    scatter_fx<TWO_D>(acc_img, E, s, v2);
            }
        }
    }
    if (own) {
        const int64_t e = e0 + q;
        if (MODE == lmh::EV_FWD) A.out[e] = r_out;
        if (MODE == lmh::EV_DATA || MODE == lmh::EV_YINIT) A.y[e] = r_y;
        if (MODE == lmh::EV_DATA_FX1 || MODE == lmh::EV_YINIT_FX1) {
            A.y[e] = r_y;
            A.out[e] = r_out;
        }
    }
}

// Event kernel.  A warp takes chunks of up to `chunk` consecutive events; the
// lanes load them coalesced and each lane sets up the traversal of its own
// event.  Groups of G lanes then process one event each (32/G events in
// flight per warp): lane s of a group takes planes i0 + s, i0 + s + G, ...,
// fetching the event's parameters from the owning lane by shuffles.
template <int MODE, bool TWO_D, int G>
__global__ void __launch_bounds__(256, G == 8 ? 2 : 3) ev_kernel(const EvArgs A)
{
    using T = ModeTraits<MODE>;
    constexpr int NG = 32 / G;
    constexpr int PC = Cache<TWO_D, G>::passes;
    extern __shared__ float s_tab[];
    int64_t eb = A.e_begin, ee = A.e_end;
    if (A.seq != nullptr) {
        const int sel = A.seq[A.u];
        if (sel >= A.n_subsets) {
            if (T::prior_branch && !A.prior_fused) prior_dual(A);
            return;
        }
        if (A.prior_only) return;
        eb = A.sub_off[sel];
        ee = A.sub_off[sel + 1];
    }
    const Geo& Gm = A.G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
    const int tofmode = Gm.tof_on ? TOF_BIN : TOF_NONE;
    const bool has_yf = A.x_yf != nullptr || A.acc_yf != nullptr || A.acci_yf != nullptr;
    const float* tab = nullptr;
    float inv_dt = 0.0f;
    if (T::traverse && A.tof_tab != nullptr && tofmode == TOF_BIN) {
        for (int k = threadIdx.x; k <= lmh::TOF_TAB_N; k += blockDim.x) s_tab[k] = A.tof_tab[k];
        __syncthreads();
        tab = s_tab;
        inv_dt = (float)lmh::TOF_TAB_N / (2.0f * Gm.W);
    }
    const int CH = A.chunk;
    const int64_t count = ee - eb;
    const int64_t nchunks = count > 0 ? (count + CH - 1) / CH : 0;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t total_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float fx_scale = 1.0f;
    if (T::back_fx) {
        const float vmax = __uint_as_float(*A.maxbits);
        fx_scale = ldexpf(1.0f, fx_exponent(vmax, (long long)count, A.stepmax));
    }
    float wmax = 0.0f;
    unsigned long long cnt_s = 0, cnt_t = 0;
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
        event_chunk<MODE, TWO_D, G>(A, A.x_std, A.x_yf, has_yf, e0, nev, tab, inv_dt, fx_scale, wmax, cnt_s, cnt_t);
    }
    if (T::count) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cnt_s += __shfl_xor_sync(FULL, cnt_s, o);
            cnt_t += __shfl_xor_sync(FULL, cnt_t, o);
        }
        if (lane == 0 && (cnt_s | cnt_t)) {
            atomicAdd(A.acci_std, cnt_s);
            atomicAdd(A.acci_std + 1, cnt_t);
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

// Event kernels of every active frame of a batch at update u.  Work items:
// for a frame whose selection is a data subset, chunks of its events; for a
// prior selection, ranges of `vitem` voxels of its prior dual step.  Warps
// take items from one self-resetting counter; a block finds an item's frame
// in a shared prefix table.
template <int MODE, bool TWO_D, int G>
__global__ void __launch_bounds__(256, G == 8 ? 2 : 3) ev_batch_kernel(const lmh::BatchEvArgs B)
{
    using T = ModeTraits<MODE>;
    extern __shared__ float s_tab[];
    __shared__ long long s_pre[lmh::BATCH_MAX + 1];
    __shared__ long long s_eb[lmh::BATCH_MAX];
    __shared__ long long s_ee[lmh::BATCH_MAX];
    __shared__ int s_kind[lmh::BATCH_MAX];  // 0 none, 1 data, 2 prior
    __shared__ float s_fx[lmh::BATCH_MAX];
    const int cap = B.cap;
    const int par = B.u & 1;
    const int sidx = (B.slot0 + B.u) & 1;
    if (threadIdx.x < cap) {
        const int s = threadIdx.x;
        long long items = 0, eb = 0, ee = 0;
        int kind = 0;
        float fxs = 1.0f;
        if (B.active[s]) {
            const EvArgs& A = B.slots[s];
            const int sel = B.seqs[(size_t)s * B.seq_stride + B.u];
            if (sel >= A.n_subsets) {
                if (T::prior_branch && !A.prior_fused) {
                    kind = 2;
                    items = ((long long)A.G.V + B.vitem - 1) / B.vitem;
                }
            } else {
                kind = 1;
                eb = A.sub_off[sel];
                ee = A.sub_off[sel + 1];
                items = (ee - eb + A.chunk - 1) / A.chunk;
                if (T::back_fx) {
                    const float vmax = __uint_as_float(A.maxbits_base[sidx]);
                    fxs = ldexpf(1.0f, fx_exponent(vmax, ee - eb, A.stepmax));
                }
            }
        }
        s_kind[s] = kind;
        s_eb[s] = eb;
        s_ee[s] = ee;
        s_fx[s] = fxs;
        s_pre[s + 1] = items;
    }
    const float* tab = nullptr;
    float inv_dt = 0.0f;
    if (T::traverse && B.tof_tab != nullptr) {
        for (int k = threadIdx.x; k <= lmh::TOF_TAB_N; k += blockDim.x) s_tab[k] = B.tof_tab[k];
        tab = s_tab;
        inv_dt = (float)lmh::TOF_TAB_N / (2.0f * B.tof_W);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int s = 0; s < cap; ++s) s_pre[s + 1] += s_pre[s];
    }
    __syncthreads();
    const long long total = s_pre[cap];
    const int lane = threadIdx.x & 31;
    const long long total_warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (;;) {
        unsigned long long cc = 0;
        if (lane == 0) cc = atomicAdd(B.queue, 1ULL);
        const long long c = (long long)__shfl_sync(FULL, cc, 0);
        if (c >= total) break;
        int s = 0;
        while (s_pre[s + 1] <= c) ++s;
        const long long local = c - s_pre[s];
        const EvArgs& A = B.slots[s];
        if (s_kind[s] == 1) {
            const int64_t e0 = s_eb[s] + local * A.chunk;
            const int nev = (int)min((long long)A.chunk, s_ee[s] - e0);
            float wmax = 0.0f;
            unsigned long long cs = 0, ct = 0;
            const bool has_yf = A.xbyf[par] != nullptr;
            event_chunk<MODE, TWO_D, G>(A, A.xb[par], A.xbyf[par], has_yf, e0, nev, tab, inv_dt, s_fx[s], wmax, cs, ct);
            if (MODE == lmh::EV_DATA_FX1) {
                float mm = wmax;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(FULL, mm, o));
                if (lane == 0 && mm > 0.0f) atomicMax(A.maxbits_base + sidx, __float_as_uint(mm));
            }
        } else if (T::prior_branch && s_kind[s] == 2) {
            const long long j0 = local * B.vitem;
            const long long j1 = min((long long)A.G.V, j0 + B.vitem);
            prior_range(A, A.xb[par], A.wpar[B.u], j0, j1, lane, 32);
        }
    }
    __syncwarp();
    if (lane == 0) {
        const unsigned d = atomicAdd(B.done, 1u);
        if (d == (unsigned)total_warps - 1) {
            *B.queue = 0ULL;
            *B.done = 0u;
        }
    }
}

size_t ev_smem(const EvArgs& a) { return a.tof_tab ? (size_t)(lmh::TOF_TAB_N + 1) * sizeof(float) : 0; }

template <int MODE, bool TWO_D>
int launch_mode(const EvArgs& a, int grid, cudaStream_t st)
{
    switch (a.group) {
        case 8:
            ev_kernel<MODE, TWO_D, 8><<<grid, 256, ev_smem(a), st>>>(a);
            break;
        case 32:
            ev_kernel<MODE, TWO_D, 32><<<grid, 256, ev_smem(a), st>>>(a);
            break;
        default:
            ev_kernel<MODE, TWO_D, 16><<<grid, 256, ev_smem(a), st>>>(a);
            break;
    }
    lmh::count_launch();
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

template <int MODE, bool TWO_D, int G>
int occupancy_grid_g()
{
    int bps = 0;
    const size_t smem = (size_t)(lmh::TOF_TAB_N + 1) * sizeof(float);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ev_kernel<MODE, TWO_D, G>, 256, smem) != cudaSuccess ||
        bps < 1)
        bps = 1;
    return bps * lmh::num_sms();
}

template <int MODE, bool TWO_D>
int occupancy_grid()
{
    // the grid is sized for the most register-hungry group width
    return std::min(occupancy_grid_g<MODE, TWO_D, 8>(),
                    std::min(occupancy_grid_g<MODE, TWO_D, 16>(), occupancy_grid_g<MODE, TWO_D, 32>()));
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

// ---- persistent epoch of a 2D frame (one cooperative launch) ----

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;  // one second

// Grid-wide barrier of a cooperative launch with a bounded wait: thread 0
// of every block arrives on bar[0]; the last arrival clears it and advances
// the generation bar[1]; the others wait for that at most WAIT_LIMIT_NS.  A
// wait that gives up sets bit 2 of *err; every block then leaves at its
// next barrier at the latest (false).
__device__ bool grid_barrier(unsigned* bar, unsigned* err, int* s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            for (unsigned it = 0; *gen == g; ++it) {
                // the time is read every 64 polls; the wait ends after WAIT_LIMIT_NS
                if ((it & 63u) == 63u && global_ns() - t0 > WAIT_LIMIT_NS) {
                    ok = 0;
                    atomicOr(err, 4u);
                    break;
                }
            }
        }
        __threadfence();
        *s_ok = ok && ((*(volatile unsigned*)err & 4u) == 0u);
    }
    __syncthreads();
    return *s_ok != 0;
}

// The image pass of one update at voxel j of a 2D grid (float accumulators
// of both layouts, TV prior): the operations of the tiled image pass in the
// same order.
__device__ __forceinline__ void persist_voxel(const lmh::PersistArgs& P, bool data, int wp, int cur, int nxt,
                                              int64_t j)
{
    const EvArgs& A = P.ev;
    const int nx = A.G.n[0], ny = A.G.n[1];
    const int64_t V = A.G.V;
    const int ix = (int)(j % nx), iy = (int)(j / nx);
    const int64_t k = (int64_t)ix * ny + iy;  // y-fastest index
    float dz;
    if (data) {
        // 2D traversals add to the first halves of the pairs
        float ay = 0.0f;
        if (A.acc_yf != nullptr) {
            ay = A.acc_yf[2 * k] + 0.0f;
            A.acc_yf[2 * k] = 0.0f;
        }
        dz = A.acc_std[2 * j] + 0.0f;
        A.acc_std[2 * j] = 0.0f;
        dz += ay;
    } else {
        // dz_j = (K^T (w+ - w))_j, components in axis order
        const float* wc = A.w_cur[wp];
        const float* wn = A.w_nxt[wp];
        dz = 0.0f;
        int64_t o = 0;
        if (nx > 1) {
            if (ix < nx - 1) dz -= wn[o + j] - wc[o + j];
            if (ix >= 1) dz += wn[o + j - 1] - wc[o + j - 1];
            o += V;
        }
        if (ny > 1) {
            if (iy < ny - 1) dz -= wn[o + j] - wc[o + j];
            if (iy >= 1) dz += wn[o + j - nx] - wc[o + j - nx];
        }
    }
    const float x0 = P.xs[cur][j], tm = P.T[j], z0 = P.z[j];
    float zh, zl = 0.0f;
    if (P.kahan) {
        float e;
        two_sum(z0, dz, zh, e);
        zl = P.zc[j] + e;
    } else {
        zh = z0 + dz;
    }
    const float zbar = fmaf(dz, data ? P.inv_p_data : P.inv_p_prior, zh + zl);
    const float xn = fmaxf(0.0f, fmaf(-tm, zbar, x0));
    P.z[j] = zh;
    if (P.kahan) P.zc[j] = zl;
    P.xw[nxt][j] = xn;
    if (P.xyf[nxt] != nullptr) P.xyf[nxt][k] = xn;
}

template <int G>
__global__ void __launch_bounds__(256, G == 8 ? 2 : 3) persist_epoch_kernel(const lmh::PersistArgs P)
{
    extern __shared__ float s_tab[];
    __shared__ int s_ok;
    const EvArgs& A = P.ev;
    const Geo& Gm = A.G;
    const float* tab = nullptr;
    float inv_dt = 0.0f;
    if (A.tof_tab != nullptr && Gm.tof_on) {
        for (int k = threadIdx.x; k <= lmh::TOF_TAB_N; k += blockDim.x) s_tab[k] = A.tof_tab[k];
        tab = s_tab;
        inv_dt = (float)lmh::TOF_TAB_N / (2.0f * Gm.W);
    }
    if (threadIdx.x == 0) {
        s_ok = 1;
        if (P.gate != nullptr && blockIdx.x == 0) {
            // failure injection: wait (bounded) for a host flag before the first update
            const unsigned long long t0 = global_ns();
            while (*(volatile const unsigned*)P.gate == 0u) {
                if (global_ns() - t0 > WAIT_LIMIT_NS) {
                    atomicOr(P.err, 4u);
                    s_ok = 0;
                    break;
                }
                __nanosleep(1000);
            }
        }
    }
    __syncthreads();
    if (!s_ok) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gn = (int64_t)gridDim.x * blockDim.x;
    const int64_t warp_global = gt >> 5, total_warps = gn >> 5;
    const int64_t V = Gm.V;
    float wmax = 0.0f;
    unsigned long long cs = 0, ct = 0;
    for (int u = 0; u < P.count; ++u) {
        const int sel = P.seq[u];
        const int cur = (P.xpar0 + u) & 1, nxt = cur ^ 1;
        const bool data = sel < A.n_subsets;
        if (data) {
            const int64_t eb = A.sub_off[sel], ee = A.sub_off[sel + 1];
            const int CH = A.chunk;
            const int64_t nch = ee > eb ? (ee - eb + CH - 1) / CH : 0;
            for (int64_t c = warp_global; c < nch; c += total_warps) {
                const int64_t e0 = eb + c * CH;
                event_chunk<lmh::EV_DATA, true, G>(A, P.xs[cur], P.xyf[cur], P.xyf[cur] != nullptr, e0,
                                                   (int)min((int64_t)CH, ee - e0), tab, inv_dt, 1.0f, wmax, cs, ct);
            }
        } else {
            prior_range(A, P.xs[cur], A.wpar[u], 0, V, gt, gn);
        }
        if (!grid_barrier(P.bar, P.err, &s_ok)) return;
        const int wp = data ? 0 : A.wpar[u];
        for (int64_t j = gt; j < V; j += gn) persist_voxel(P, data, wp, cur, nxt, j);
        if (!grid_barrier(P.bar, P.err, &s_ok)) return;
    }
}

template <int G>
int persist_blocks()
{
    static int nb = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        const size_t smem = (size_t)(lmh::TOF_TAB_N + 1) * 4;
        cudaFuncSetAttribute(persist_epoch_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, persist_epoch_kernel<G>, 256, smem) != cudaSuccess)
            b = 0;
        nb = b;
    });
    return nb;
}

}  // namespace

namespace lmh {

bool persist_supported()
{
    static int ok = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, v = 0;
        ok = cudaGetDevice(&dev) == cudaSuccess &&
                     cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && v
                 ? 1
                 : 0;
    });
    return ok == 1;
}

// All blocks must be resident at once (cooperative launch): the SM count
// times the resident blocks per SM, 0 if none fit.
int persist_grid(int group)
{
    const int b = group == 8 ? persist_blocks<8>() : group == 32 ? persist_blocks<32>() : persist_blocks<16>();
    return b * num_sms();
}

int launch_persist_epoch(const PersistArgs& p, int group, int grid, cudaStream_t st)
{
    LM_CHECK(grid > 0, LM_ERR_CUDA, "the persistent epoch kernel does not fit on the device");
    const size_t smem = (size_t)(TOF_TAB_N + 1) * 4;
    void* args[] = {(void*)&p};
    cudaError_t e;
    switch (group) {
    case 8: e = cudaLaunchCooperativeKernel((void*)persist_epoch_kernel<8>, grid, 256, args, smem, st); break;
    case 32: e = cudaLaunchCooperativeKernel((void*)persist_epoch_kernel<32>, grid, 256, args, smem, st); break;
    default: e = cudaLaunchCooperativeKernel((void*)persist_epoch_kernel<16>, grid, 256, args, smem, st); break;
    }
    LM_CHECK(e == cudaSuccess, LM_ERR_CUDA, "persistent epoch launch failed: %s", cudaGetErrorString(e));
    count_launch();
    return LM_OK;
}

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
        LM_CASE(EV_EM)
        default:
            return LM_ERR_INVALID_ARG;
    }
#undef LM_CASE
}

template <int MODE, bool TWO_D>
int launch_batch_mode(int group, const BatchEvArgs& b, int grid, cudaStream_t st)
{
    const size_t smem = b.tof_tab ? (size_t)(TOF_TAB_N + 1) * sizeof(float) : 0;
    switch (group) {
        case 8:
            ev_batch_kernel<MODE, TWO_D, 8><<<grid, 256, smem, st>>>(b);
            break;
        case 32:
            ev_batch_kernel<MODE, TWO_D, 32><<<grid, 256, smem, st>>>(b);
            break;
        default:
            ev_batch_kernel<MODE, TWO_D, 16><<<grid, 256, smem, st>>>(b);
            break;
    }
    count_launch();
    return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

int launch_events_batch(int mode, bool two_d, int group, const BatchEvArgs& b, int grid, cudaStream_t st)
{
    switch (mode) {
        case EV_DATA:
            return two_d ? launch_batch_mode<EV_DATA, true>(group, b, grid, st)
                         : launch_batch_mode<EV_DATA, false>(group, b, grid, st);
        case EV_DATA_FX1:
            return two_d ? launch_batch_mode<EV_DATA_FX1, true>(group, b, grid, st)
                         : launch_batch_mode<EV_DATA_FX1, false>(group, b, grid, st);
        case EV_BACK_FX:
            return two_d ? launch_batch_mode<EV_BACK_FX, true>(group, b, grid, st)
                         : launch_batch_mode<EV_BACK_FX, false>(group, b, grid, st);
        default:
            return LM_ERR_INVALID_ARG;
    }
}

template <int MODE, bool TWO_D>
int batch_occupancy(int group)
{
    int g = 1 << 30;
    const size_t smem = (size_t)(TOF_TAB_N + 1) * sizeof(float);
    int bps = 0;
    if ((group == 8 || group == 0) &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ev_batch_kernel<MODE, TWO_D, 8>, 256, smem) == cudaSuccess)
        g = std::min(g, std::max(1, bps));
    if ((group == 16 || group == 0) &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ev_batch_kernel<MODE, TWO_D, 16>, 256, smem) == cudaSuccess)
        g = std::min(g, std::max(1, bps));
    if ((group == 32 || group == 0) &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ev_batch_kernel<MODE, TWO_D, 32>, 256, smem) == cudaSuccess)
        g = std::min(g, std::max(1, bps));
    if (g == (1 << 30)) g = 1;
    return g * num_sms();
}

int ev_batch_grid(int mode, bool two_d, int group)
{
    switch (mode) {
        case EV_DATA:
            return two_d ? batch_occupancy<EV_DATA, true>(group) : batch_occupancy<EV_DATA, false>(group);
        case EV_DATA_FX1:
            return two_d ? batch_occupancy<EV_DATA_FX1, true>(group) : batch_occupancy<EV_DATA_FX1, false>(group);
        case EV_BACK_FX:
            return two_d ? batch_occupancy<EV_BACK_FX, true>(group) : batch_occupancy<EV_BACK_FX, false>(group);
        default:
            return num_sms();
    }
}

template <int MODE, bool TWO_D>
int occupancy_grid_for(int group)
{
    switch (group) {
        case 8:
            return occupancy_grid_g<MODE, TWO_D, 8>();
        case 32:
            return occupancy_grid_g<MODE, TWO_D, 32>();
        case 16:
            return occupancy_grid_g<MODE, TWO_D, 16>();
        default:
            return occupancy_grid<MODE, TWO_D>();
    }
}

// Resident blocks x SMs of the event kernel with `group` lanes per event.
int ev_grid_g(int mode, bool two_d, int group)
{
#define LM_CASE(M) \
    case M:        \
        return two_d ? occupancy_grid_for<M, true>(group) : occupancy_grid_for<M, false>(group);
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
        LM_CASE(EV_EM)
        default:
            return num_sms();
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
        LM_CASE(EV_EM)
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

int lm_struct_sizes(size_t* out, int n)
{
    const size_t sz[6] = {sizeof(lm_scanner), sizeof(lm_grid),   sizeof(lm_tof),
                          sizeof(lm_events),  sizeof(lm_params), sizeof(lm_server_config)};
    for (int i = 0; out != nullptr && i < n && i < 6; ++i) out[i] = sz[i];
    return 6;
}

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


}  // extern "C"
