// Device-side geometry of the listmode TOF Joseph projector (sm_103a).
//
// One event (or LOR) is processed by a group of 32 lanes (one warp); lane l
// takes the voxel planes i0 + l, i0 + l + 32, ... along the principal axis,
// so that the 32 gathers/atomics of one instruction touch consecutive voxels
// of the image row that runs along that axis.  Images are kept in two
// layouts during the iteration: x-fastest ("std") for LORs whose principal
// axis is x or z, y-fastest ("yf", index (iz*nx + ix)*ny + iy) for LORs
// whose principal axis is y, so both families read along contiguous rows.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lmk {

constexpr unsigned FULL = 0xffffffffu;

struct Geo {
    int n[3];
    float h[3];
    float o[3];
    int tof_on;      // n_bins > 0
    int M;           // (n_bins-1)/2
    float bin;       // TOF bin width (mm)
    float W;         // n_sigma * sigma (mm)
    float inv_s;     // 1 / (sqrt(2) sigma)
    const float* xtal;
    int n_det;
    int V;
};

enum TofMode { TOF_NONE = 0, TOF_BIN = 1, TOF_SUM = 2 };

// Traversal of one LOR: affine descriptions in the plane index i.
struct Lor {
    int i0, cnt;          // planes [i0, i0+cnt)
    float ua0, sa;        // secondary axis A coordinate (voxel units) = ua0 + i*sa
    float ub0, sb;        // secondary axis B
    float tau0, dtau;     // TOF coordinate relative to the bin centre (mm)
    float step;           // sample length (mm)
    int sk, sA, sB;       // voxel strides of the plane index and the secondary axes
    int nA, nB;
    int yf;               // 1: use the y-fastest image (principal axis y)
    int k;                // principal axis
};

__device__ __forceinline__ float sel3(int k, float a, float b, float c) { return k == 0 ? a : (k == 1 ? b : c); }
__device__ __forceinline__ int sel3i(int k, int a, int b, int c) { return k == 0 ? a : (k == 1 ? b : c); }

// Sets up the traversal; returns false if the LOR has no candidate sample.
// m: signed TOF bin (ignored unless tofmode == TOF_BIN).
__device__ __forceinline__ bool lor_setup(const Geo& G, int d1, int d2, int m, int tofmode, bool has_yf,
                                          Lor& L)
{
    const float* A = G.xtal + 3 * d1;
    const float* B = G.xtal + 3 * d2;
    const float a0 = __ldg(A), a1 = __ldg(A + 1), a2 = __ldg(A + 2);
    const float d0 = __ldg(B) - a0, dd1 = __ldg(B + 1) - a1, dd2 = __ldg(B + 2) - a2;
    int k = 0;
    float adk = fabsf(d0);
    if (fabsf(dd1) > adk) { k = 1; adk = fabsf(dd1); }
    if (fabsf(dd2) > adk) { k = 2; adk = fabsf(dd2); }
    if (adk == 0.0f) return false;
    const int ka = (k == 0) ? 1 : 0;
    const int kb = (k == 2) ? 1 : 2;
    L.k = k;
    const float dk = sel3(k, d0, dd1, dd2);
    const float da = sel3(ka, d0, dd1, dd2), db = sel3(kb, d0, dd1, dd2);
    // line centre c = a + d/2; plane i: mu_i = (o_k + i h_k - c_k)/d_k, point c + mu_i d
    const float ck = fmaf(0.5f, dk, sel3(k, a0, a1, a2));
    const float ca = fmaf(0.5f, da, sel3(ka, a0, a1, a2));
    const float cb = fmaf(0.5f, db, sel3(kb, a0, a1, a2));
    const float hk = sel3(k, G.h[0], G.h[1], G.h[2]);
    const float ha = sel3(ka, G.h[0], G.h[1], G.h[2]);
    const float hb = sel3(kb, G.h[0], G.h[1], G.h[2]);
    const float ok = sel3(k, G.o[0], G.o[1], G.o[2]);
    const float oa = sel3(ka, G.o[0], G.o[1], G.o[2]);
    const float ob = sel3(kb, G.o[0], G.o[1], G.o[2]);
    const float inv = 1.0f / dk;
    const float mu0 = (ok - ck) * inv;
    const float dmu = hk * inv;
    const float Llen = sqrtf(fmaf(d0, d0, fmaf(dd1, dd1, dd2 * dd2)));
    L.ua0 = (fmaf(mu0, da, ca) - oa) / ha;
    L.sa = dmu * da / ha;
    L.ub0 = (fmaf(mu0, db, cb) - ob) / hb;
    L.sb = dmu * db / hb;
    L.step = hk * Llen * fabsf(inv);
    L.tau0 = mu0 * Llen;
    if (tofmode == TOF_BIN) L.tau0 -= (float)m * G.bin;
    L.dtau = dmu * Llen;
    const int nk = sel3i(k, G.n[0], G.n[1], G.n[2]);
    L.nA = sel3i(ka, G.n[0], G.n[1], G.n[2]);
    L.nB = sel3i(kb, G.n[0], G.n[1], G.n[2]);
    const int nx = G.n[0], ny = G.n[1];
    if (k == 0) {
        L.sk = 1; L.sA = nx; L.sB = nx * ny; L.yf = 0;
    } else if (k == 1) {
        if (has_yf) { L.sk = 1; L.sA = ny; L.sB = nx * ny; L.yf = 1; }
        else { L.sk = nx; L.sA = 1; L.sB = nx * ny; L.yf = 0; }
    } else {
        L.sk = nx * ny; L.sA = 1; L.sB = nx; L.yf = 0;
    }
    // candidate plane range: inside [0, nk-1], secondary coordinates in
    // (-1, n) and (for TOF) |tau| <= W; widened by one plane on each side,
    // the per-sample tests decide.
    float lo = 0.0f, hi = (float)(nk - 1);
    auto clip = [&](float u0, float s, float ulo, float uhi) {
        if (s == 0.0f) {
            if (!(u0 > ulo && u0 < uhi)) { lo = 1.0f; hi = 0.0f; }
        } else {
            float t0 = (ulo - u0) / s, t1 = (uhi - u0) / s;
            lo = fmaxf(lo, fminf(t0, t1) - 1.0f);
            hi = fminf(hi, fmaxf(t0, t1) + 1.0f);
        }
    };
    clip(L.ua0, L.sa, -1.0f, (float)L.nA);
    clip(L.ub0, L.sb, -1.0f, (float)L.nB);
    if (tofmode == TOF_BIN) clip(L.tau0, L.dtau, -G.W, G.W);
    if (!(lo <= hi)) return false;
    const int i0 = (int)fmaxf(0.0f, floorf(lo));
    const int i1 = (int)fminf((float)(nk - 1), ceilf(hi));
    L.i0 = i0;
    L.cnt = i1 - i0 + 1;
    return L.cnt > 0;
}

// TOF weight of a sample.  TOF_BIN: bin-integrated Gaussian of the event's
// bin, 0 outside the truncation window.  TOF_SUM: sum over all bins whose
// window contains the sample; the bin integrals telescope to one difference.
__device__ __forceinline__ float tof_weight(const Geo& G, int tofmode, float tau)
{
    if (tofmode == TOF_BIN) {
        if (fabsf(tau) > G.W) return 0.0f;
        const float hb = 0.5f * G.bin;
        return 0.5f * (erff((tau + hb) * G.inv_s) - erff((tau - hb) * G.inv_s));
    }
    if (tofmode == TOF_SUM) {
        // bins m with |tau - m bin| <= W, m in [-M, M]
        const float mlo = fmaxf((float)(-G.M), ceilf((tau - G.W) / G.bin));
        const float mhi = fminf((float)G.M, floorf((tau + G.W) / G.bin));
        if (mlo > mhi) return 0.0f;
        const float hb = 0.5f * G.bin;
        return 0.5f * (erff((tau - fmaf(mlo, G.bin, -hb)) * G.inv_s) -
                       erff((tau - fmaf(mhi, G.bin, hb)) * G.inv_s));
    }
    return 1.0f;
}

// One sample: base voxel index and the (up to) four bilinear weights times
// TOF weight times sample length; invalid neighbours carry weight 0.
struct Smp {
    int base;
    float w0, w1, w2, w3;  // (A, B), (A+1, B), (A, B+1), (A+1, B+1)
};

template <bool TWO_D>
__device__ __forceinline__ bool sample_at(const Geo& G, const Lor& L, int tofmode, int i, Smp& s)
{
    const float fi = (float)i;
    float wt = L.step;
    if (tofmode != TOF_NONE) {
        const float tau = fmaf(fi, L.dtau, L.tau0);
        wt *= tof_weight(G, tofmode, tau);
        if (wt == 0.0f) return false;
    }
    const float ua = fmaf(fi, L.sa, L.ua0);
    const float fla = floorf(ua);
    const int ia = (int)fla;
    const float fa = ua - fla;
    const float wa0 = (ia >= 0 && ia < L.nA) ? (1.0f - fa) : 0.0f;
    const float wa1 = (ia + 1 >= 0 && ia + 1 < L.nA) ? fa : 0.0f;
    if (TWO_D) {
        // 2D grids: the third axis has one voxel and the LOR lies in its plane
        s.base = i * L.sk + ia * L.sA;
        s.w0 = wt * wa0;
        s.w1 = wt * wa1;
        s.w2 = 0.0f;
        s.w3 = 0.0f;
        return (wa0 != 0.0f) || (wa1 != 0.0f);
    } else {
        const float ub = fmaf(fi, L.sb, L.ub0);
        const float flb = floorf(ub);
        const int ib = (int)flb;
        const float fb = ub - flb;
        const float wb0 = (ib >= 0 && ib < L.nB) ? (1.0f - fb) : 0.0f;
        const float wb1 = (ib + 1 >= 0 && ib + 1 < L.nB) ? fb : 0.0f;
        s.base = i * L.sk + ia * L.sA + ib * L.sB;
        s.w0 = wt * wa0 * wb0;
        s.w1 = wt * wa1 * wb0;
        s.w2 = wt * wa0 * wb1;
        s.w3 = wt * wa1 * wb1;
        return (s.w0 != 0.0f) || (s.w1 != 0.0f) || (s.w2 != 0.0f) || (s.w3 != 0.0f);
    }
}

template <bool TWO_D>
__device__ __forceinline__ float gather(const float* __restrict__ img, const Lor& L, const Smp& s)
{
    float v = 0.0f;
    if (s.w0 != 0.0f) v = fmaf(s.w0, __ldg(img + s.base), v);
    if (s.w1 != 0.0f) v = fmaf(s.w1, __ldg(img + s.base + L.sA), v);
    if (!TWO_D) {
        if (s.w2 != 0.0f) v = fmaf(s.w2, __ldg(img + s.base + L.sB), v);
        if (s.w3 != 0.0f) v = fmaf(s.w3, __ldg(img + s.base + L.sA + L.sB), v);
    }
    return v;
}

template <bool TWO_D>
__device__ __forceinline__ float wsum(const Smp& s)
{
    return TWO_D ? (s.w0 + s.w1) : ((s.w0 + s.w1) + (s.w2 + s.w3));
}

template <bool TWO_D>
__device__ __forceinline__ void scatter(float* img, const Lor& L, const Smp& s, float val)
{
    if (s.w0 != 0.0f) atomicAdd(img + s.base, s.w0 * val);
    if (s.w1 != 0.0f) atomicAdd(img + s.base + L.sA, s.w1 * val);
    if (!TWO_D) {
        if (s.w2 != 0.0f) atomicAdd(img + s.base + L.sB, s.w2 * val);
        if (s.w3 != 0.0f) atomicAdd(img + s.base + L.sA + L.sB, s.w3 * val);
    }
}

// Scatter into a z-paired accumulator: element 2j holds voxel j, element
// 2j + 1 voxel j + nx*ny.  For principal axes x and y the second secondary
// axis is z, so a sample's two z-neighbours share one 8-byte pair and one
// vector atomic instead of two scattered scalar ones (half the L2 sector
// operations); z-principal and 2D traversals add to the first elements.
template <bool TWO_D>
__device__ __forceinline__ void scatter_pairs(float* ap, const Lor& L, const Smp& s, float val)
{
    if (TWO_D || L.k == 2) {
        if (s.w0 != 0.0f) atomicAdd(ap + 2 * (int64_t)s.base, s.w0 * val);
        if (s.w1 != 0.0f) atomicAdd(ap + 2 * ((int64_t)s.base + L.sA), s.w1 * val);
        if (!TWO_D) {
            if (s.w2 != 0.0f) atomicAdd(ap + 2 * ((int64_t)s.base + L.sB), s.w2 * val);
            if (s.w3 != 0.0f) atomicAdd(ap + 2 * ((int64_t)s.base + L.sA + L.sB), s.w3 * val);
        }
        return;
    }
    float2* p2 = reinterpret_cast<float2*>(ap);
    if (s.w0 != 0.0f || s.w1 != 0.0f) {
        // the base slice is inside the grid (its z weight is non-zero)
        if (s.w0 != 0.0f || s.w2 != 0.0f) atomicAdd(p2 + s.base, make_float2(s.w0 * val, s.w2 * val));
        if (s.w1 != 0.0f || s.w3 != 0.0f) atomicAdd(p2 + s.base + L.sA, make_float2(s.w1 * val, s.w3 * val));
    } else {
        // base slice -1: only the neighbours in slice 0
        if (s.w2 != 0.0f) atomicAdd(ap + 2 * ((int64_t)s.base + L.sB), s.w2 * val);
        if (s.w3 != 0.0f) atomicAdd(ap + 2 * ((int64_t)s.base + L.sA + L.sB), s.w3 * val);
    }
}

// Fixed-point scatter: value * weight * 2^E rounded to the nearest integer,
// added with 64-bit integer atomics (order-independent, exact).
__device__ __forceinline__ void fx_add(unsigned long long* p, float q)
{
    const long long iv = __float2ll_rn(q);
    if (iv != 0) atomicAdd(p, (unsigned long long)iv);
}

template <bool TWO_D>
__device__ __forceinline__ void scatter_fx(unsigned long long* img, const Lor& L, const Smp& s, float val2E)
{
    if (s.w0 != 0.0f) fx_add(img + s.base, s.w0 * val2E);
    if (s.w1 != 0.0f) fx_add(img + s.base + L.sA, s.w1 * val2E);
    if (!TWO_D) {
        if (s.w2 != 0.0f) fx_add(img + s.base + L.sB, s.w2 * val2E);
        if (s.w3 != 0.0f) fx_add(img + s.base + L.sA + L.sB, s.w3 * val2E);
    }
}

// Factor of the projection onto the ball of radius beta (the prox of R^*
// for the isotropic TV, Sec. "Numerical experiments"):
// w+ = v / max(1, |v|/beta) = v * tv_ball_scale(|v|^2, beta); beta = 0 gives
// w+ = 0.  One reciprocal square root instead of a square root and divisions.
__device__ __forceinline__ float tv_ball_scale(float n2, float beta)
{
    return n2 > beta * beta ? beta * rsqrtf(n2) : 1.0f;
}

// Directional TV (Sec. "Numerical experiments"): the part of a difference
// vector (gx, gy, gz) perpendicular to the structural field (fx, fy, fz) of
// the voxel, g - f (f . g); components of axes of length 1 are 0 in both.
__device__ __forceinline__ void dtv_perp(float fx, float fy, float fz, float& gx, float& gy, float& gz)
{
    const float s = fmaf(fx, gx, fmaf(fy, gy, fz * gz));
    gx = fmaf(-fx, s, gx);
    gy = fmaf(-fy, s, gy);
    gz = fmaf(-fz, s, gz);
}

// Sum a + b with its exact rounding error (TwoSum, Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Closed-form proximal map of the Poisson conjugate with data 1 and step
// t = mu*S (Eq. proxD with the listmode rescaling of the appendix):
//   1/2 (a + 1 - sqrt((a-1)^2 + 4t)).
// For a >= 1 the algebraically equal 2(a - t)/(a + 1 + sqrt(.)) avoids the
// cancellation between a + 1 and the root.
__device__ __forceinline__ float prox_dstar(float a, float t)
{
    const float am1 = a - 1.0f;
    const float r = sqrtf(fmaf(am1, am1, 4.0f * t));
    if (a >= 1.0f) return 2.0f * (a - t) / (a + 1.0f + r);
    return 0.5f * (a + 1.0f - r);
}

// Fixed-point exponent for a deterministic back-projection: every voxel sum
// is bounded by count * vmax * stepmax (one contribution per event and
// voxel, weights <= 1), which is kept below 2^62.
__device__ __forceinline__ int fx_exponent(float vmax, long long count, float stepmax)
{
    const double bound = (double)vmax * (double)stepmax * (double)(count > 0 ? count : 1);
    if (!(bound > 0.0)) return 0;
    int ex;
    frexp(bound, &ex);  // bound < 2^ex
    int E = 62 - ex;
    if (E > 120) E = 120;
    if (E < -120) E = -120;
    return E;
}

}  // namespace lmk
