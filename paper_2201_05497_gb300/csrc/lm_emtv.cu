// Listmode EM-TV (Alg. 3): the warm start of the listmode experiments.  One
// pass over the n subsets; per subset a listmode EM step on the subset's
// events (the event kernel in its EM mode, scattering c_e / (c_e J_e x + s_e))
// followed by a weighted TV denoising problem
//   x = argmin_{u >= 0} sum_j w_j/2 (u_j - z_j)^2 + ||K u||_{2,1},  w = g / (beta x),
// solved by the accelerated primal-dual algorithm of Chambolle & Pock (2011,
// their Alg. 2) with G(u) = sum_j w_j/2 (u_j - z_j)^2 + i_{u >= 0}, uniformly
// convex with modulus gam = min_j w_j over the free voxels, and F^* the
// indicator of the unit 2-norm balls.
//
// One inner iteration is two voxel passes (dual, primal).  The step-size schedule
// (tau_k, sigma_k, theta_k) depends only on gam and ||K||; one thread computes
// it in FP64 on the device once gam is known, so the whole epoch is queued
// on the stream without a host round trip.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "lm_internal.h"

using namespace lmk;
using namespace lmh;

namespace {

constexpr int EMTV_MAX_ITERS = 10000;

struct Sched {
    // ~(float bits) of min w over the free voxels: non-negative floats order
    // as unsigned integers, so the minimum is an atomic maximum of the
    // complements and a cleared word (0) means "no free voxel"
    unsigned gam_nbits;
    unsigned done;             // the event kernel's self-resetting work counters
    unsigned long long queue;
    unsigned pad[60];
    float tau[EMTV_MAX_ITERS];
    float sigma[EMTV_MAX_ITERS];
    float theta[EMTV_MAX_ITERS];
};

struct Ws {
    float* z;
    float* w;
    float* ubar;   // extrapolated primal iterate
    float* q;      // dual iterate [ndim][V]
    float* pair_std; // the EM back-projection's (voxel j, voxel j + nx*ny) float pairs, x-fastest
    float* pair_yf;  // the same, y-fastest (both zero between steps: the fold clears them)
    float* x_yf;   // y-fastest copy of x for the EM gathers
    float* tof_tab; // the TOF kernel tabulated for the event kernel (TOF_TAB_N + 1 floats)
    Sched* sc;
};

struct Axes {
    int nd;
    int n[3];
    int64_t st[3];  // strides of the TV components' axes
    int dim[3];     // grid dimension of component c
};

Axes axes_of(const lm_grid* g)
{
    Axes a;
    std::memset(&a, 0, sizeof(a));
    const int64_t stride[3] = {1, g->n[0], (int64_t)g->n[0] * g->n[1]};
    for (int d = 0; d < 3; ++d)
        if (g->n[d] > 1) {
            a.n[a.nd] = g->n[d];
            a.st[a.nd] = stride[d];
            a.dim[a.nd] = d;
            ++a.nd;
        }
    return a;
}

size_t ws_layout(const lm_grid* g, Ws* w, void* base)
{
    const size_t V = (size_t)nvox(g);
    const int nd = std::max(1, axes_of(g).nd);
    char* p = (char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* r = p ? p + off : nullptr;
        off += align_up(bytes);
        return r;
    };
    Ws t;
    t.z = (float*)take(V * 4);
    t.w = (float*)take(V * 4);
    t.ubar = (float*)take(V * 4);
    t.q = (float*)take((size_t)nd * V * 4);
    t.pair_std = (float*)take(2 * V * 4);
    t.pair_yf = (float*)take(2 * V * 4);
    t.x_yf = (float*)take(V * 4);
    t.tof_tab = (float*)take((size_t)(TOF_TAB_N + 1) * 4);
    t.sc = (Sched*)take(sizeof(Sched));
    if (w) *w = t;
    return off;
}

// z_j = x_j n / g_j * b_j (0 where g_j = 0), b = the EM back-projection.
// With a prior (beta > 0) also the weights and the start of the inner
// problem: free_j = x_j > 0 and g_j > 0; w_j = g_j / (beta x_j) (0 = held);
// u = ubar = z on free voxels, 0 elsewhere (u written to x); q = 0; gam.
// Without a prior x = z.
__global__ void __launch_bounds__(256) em_fold_kernel(float* __restrict__ x, float* __restrict__ z,
                                                      const float* __restrict__ sens, float* __restrict__ w,
                                                      float* __restrict__ ubar, float* __restrict__ q, int nd,
                                                      int64_t V, float n_sub, float beta, Sched* sc)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const float xj = x[j], gj = sens[j];
        const float zj = gj > 0.0f ? xj * n_sub / gj * z[j] : 0.0f;
        if (!(beta > 0.0f)) {
            x[j] = zj;
            continue;
        }
        z[j] = zj;
        const bool fr = xj > 0.0f && gj > 0.0f;
        const float wj = fr ? gj / (beta * xj) : 0.0f;
        w[j] = wj;
        const float u0 = fr ? zj : 0.0f;
        x[j] = u0;
        ubar[j] = u0;
        for (int c = 0; c < nd; ++c) q[c * V + j] = 0.0f;
        if (fr) atomicMax(&sc->gam_nbits, ~__float_as_uint(wj));
    }
}

// Start of a standalone denoising call: free_j = w_j > 0.
__global__ void __launch_bounds__(256) denoise_init_kernel(const float* __restrict__ z, const float* __restrict__ w,
                                                           float* __restrict__ u, float* __restrict__ ubar,
                                                           float* __restrict__ q, int nd, int64_t V, Sched* sc)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x) {
        const float wj = w[j];
        const bool fr = wj > 0.0f;
        const float u0 = fr ? z[j] : 0.0f;
        u[j] = u0;
        ubar[j] = u0;
        for (int c = 0; c < nd; ++c) q[c * V + j] = 0.0f;
        if (fr) atomicMax(&sc->gam_nbits, ~__float_as_uint(wj));
    }
}

// The bin-integrated Gaussian TOF weight w(tau) on TOF_TAB_N intervals of
// [-W, W] (the table the event kernel interpolates), evaluated in FP64.
__global__ void tof_tab_kernel(float* tab, double W, double D, double s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > TOF_TAB_N) return;
    const double tau = -W + 2.0 * W * k / TOF_TAB_N;
    tab[k] = (float)(0.5 * (erf((tau + 0.5 * D) / s) - erf((tau - 0.5 * D) / s)));
}

// Clears the work counters and the pair accumulators and tabulates the TOF
// kernel for the EM steps.
int em_prepare(const lm_grid* grid, const lm_tof* tof, const Ws& W, cudaStream_t st)
{
    LM_CUDA(cudaMemsetAsync(W.sc, 0, 16, st));
    const size_t V = (size_t)nvox(grid);
    LM_CUDA(cudaMemsetAsync(W.pair_std, 0, 2 * V * 4, st));
    LM_CUDA(cudaMemsetAsync(W.pair_yf, 0, 2 * V * 4, st));
    if (tof->n_bins > 0) {
        const double sig = tof->sigma_mm;
        tof_tab_kernel<<<(TOF_TAB_N + 256) / 256, 256, 0, st>>>(W.tof_tab, (double)tof->n_sigma * sig,
                                                                (double)tof->bin_mm, std::sqrt(2.0) * sig);
        count_launch();
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}

// Step sizes of the accelerated algorithm: tau_0 = sigma_0 = 0.99 / ||K||;
// theta_k = 1 / sqrt(1 + 2 gam tau_k); tau_{k+1} = theta_k tau_k;
// sigma_{k+1} = sigma_k / theta_k (so tau_k sigma_k ||K||^2 stays 0.99^2).
__global__ void sched_kernel(Sched* sc, int iters, double knorm)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const unsigned nb = sc->gam_nbits;
    const double gam = nb == 0u ? 0.0 : (double)__uint_as_float(~nb);
    double tau = 0.99 / knorm, sigma = 0.99 / knorm;
    for (int k = 0; k < iters; ++k) {
        const double th = 1.0 / sqrt(1.0 + 2.0 * gam * tau);
        sc->tau[k] = (float)tau;
        sc->sigma[k] = (float)sigma;
        sc->theta[k] = (float)th;
        tau *= th;
        sigma /= th;
    }
}

// One inner iteration is two voxel passes: the dual step needs the forward
// neighbours of ubar, the primal step the backward neighbours of the new q,
// so the second pass starts when the first has finished.  Each thread takes
// four consecutive voxels of one image row with 16-byte loads when rows are
// a multiple of 4 long (all loads issued before any arithmetic), else one
// voxel.  Indices are 32-bit (grids have fewer than 2^31 voxels).
struct PdArgs {
    float* ubar;
    float* q;            // [ndim][V]
    float* u;
    const float* z;
    const float* w;
    int nx, ny, nz;
    int cx, cy, cz;      // component of the x, y, z difference (-1: axis of length 1)
    int V;
    const Sched* sc;
    int k;
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
__device__ __forceinline__ void st4(float* p, const float* v) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }

// q <- proj_{|.| <= 1}(q + sigma_k K ubar) at voxel j (components in axis
// order), from ubar_j and its forward neighbours.
__device__ __forceinline__ void dual_point(const PdArgs& A, float sg, float u0, float ux, float uy, float uz, bool inx,
                                           bool iny, bool inz, float q0, float q1, float q2, float& o0, float& o1,
                                           float& o2)
{
    float vx = 0.0f, vy = 0.0f, vz = 0.0f, n2 = 0.0f;
    if (A.cx >= 0) {
        vx = fmaf(sg, inx ? ux - u0 : 0.0f, q0);
        n2 = fmaf(vx, vx, n2);
    }
    if (A.cy >= 0) {
        vy = fmaf(sg, iny ? uy - u0 : 0.0f, q1);
        n2 = fmaf(vy, vy, n2);
    }
    if (A.cz >= 0) {
        vz = fmaf(sg, inz ? uz - u0 : 0.0f, q2);
        n2 = fmaf(vz, vz, n2);
    }
    const float s = tv_ball_scale(n2, 1.0f);
    o0 = __fmul_rn(vx, s);
    o1 = __fmul_rn(vy, s);
    o2 = __fmul_rn(vz, s);
}

// u+ = prox_{tau G}(u - tau K^T q) = max(0, (v + tau w z) / (1 + tau w)) on
// free voxels (0 on held ones); returns u+, ubar+ = u+ + theta (u+ - u).
__device__ __forceinline__ float primal_point(float tau, float th, float kt, float uj, float wj, float zj, float& ub)
{
    float un = 0.0f;
    if (wj > 0.0f) {
        const float v = fmaf(-tau, kt, uj);
        const float tw = tau * wj;
        un = fmaxf(0.0f, fmaf(tw, zj, v) / (1.0f + tw));
    }
    ub = fmaf(th, un - uj, un);
    return un;
}

__global__ void __launch_bounds__(256) dual_quad_kernel(const PdArgs A)
{
    const int nq = A.nx >> 2;
    const int nquads = A.V >> 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nquads) return;
    const float sg = A.sc->sigma[A.k];
    const int nx = A.nx, ny = A.ny, nz = A.nz, V = A.V;
    const int ix = (t % nq) * 4, r = t / nq, iy = r % ny, iz = r / ny;
    const int j = r * nx + ix;
    const bool iny = iy < ny - 1, inz = iz < nz - 1;
    const float4 uc = ld4(A.ubar + j);
    const float ur = (A.cx >= 0 && ix + 4 < nx) ? A.ubar[j + 4] : 0.0f;
    const float4 uy = (A.cy >= 0 && iny) ? ld4(A.ubar + j + nx) : uc;
    const float4 uz = (A.cz >= 0 && inz) ? ld4(A.ubar + j + nx * ny) : uc;
    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 qx = A.cx >= 0 ? ld4(A.q + A.cx * V + j) : zero;
    const float4 qy = A.cy >= 0 ? ld4(A.q + A.cy * V + j) : zero;
    const float4 qz = A.cz >= 0 ? ld4(A.q + A.cz * V + j) : zero;
    float ox[4], oy[4], oz[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        dual_point(A, sg, f4(uc, i), i < 3 ? f4(uc, i + 1) : ur, f4(uy, i), f4(uz, i), ix + i < nx - 1, iny, inz,
                   f4(qx, i), f4(qy, i), f4(qz, i), ox[i], oy[i], oz[i]);
    if (A.cx >= 0) st4(A.q + A.cx * V + j, ox);
    if (A.cy >= 0) st4(A.q + A.cy * V + j, oy);
    if (A.cz >= 0) st4(A.q + A.cz * V + j, oz);
}

__global__ void __launch_bounds__(256) primal_quad_kernel(const PdArgs A)
{
    const int nq = A.nx >> 2;
    const int nquads = A.V >> 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nquads) return;
    const float tau = A.sc->tau[A.k], th = A.sc->theta[A.k];
    const int nx = A.nx, ny = A.ny, nz = A.nz, V = A.V;
    const int ix = (t % nq) * 4, r = t / nq, iy = r % ny, iz = r / ny;
    const int j = r * nx + ix;
    const int sz = nx * ny;
    const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4 qx = A.cx >= 0 ? ld4(A.q + A.cx * V + j) : zero;
    const float qxl = (A.cx >= 0 && ix >= 1) ? A.q[A.cx * V + j - 1] : 0.0f;
    const float4 qy = A.cy >= 0 ? ld4(A.q + A.cy * V + j) : zero;
    const float4 qyb = (A.cy >= 0 && iy >= 1) ? ld4(A.q + A.cy * V + j - nx) : zero;
    const float4 qz = A.cz >= 0 ? ld4(A.q + A.cz * V + j) : zero;
    const float4 qzb = (A.cz >= 0 && iz >= 1) ? ld4(A.q + A.cz * V + j - sz) : zero;
    const float4 u4 = ld4(A.u + j), w4 = ld4(A.w + j), z4 = ld4(A.z + j);
    float uo[4], bo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float kt = 0.0f;  // (K^T q)_j, components in axis order
        if (A.cx >= 0) {
            if (ix + i < nx - 1) kt -= f4(qx, i);
            if (ix + i >= 1) kt += i > 0 ? f4(qx, i - 1) : qxl;
        }
        if (A.cy >= 0) {
            if (iy < ny - 1) kt -= f4(qy, i);
            if (iy >= 1) kt += f4(qyb, i);
        }
        if (A.cz >= 0) {
            if (iz < nz - 1) kt -= f4(qz, i);
            if (iz >= 1) kt += f4(qzb, i);
        }
        uo[i] = primal_point(tau, th, kt, f4(u4, i), f4(w4, i), f4(z4, i), bo[i]);
    }
    st4(A.u + j, uo);
    st4(A.ubar + j, bo);
}

// One voxel per thread (rows not a multiple of 4 long).
__global__ void __launch_bounds__(256) dual_point_kernel(const PdArgs A)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.V) return;
    const float sg = A.sc->sigma[A.k];
    const int nx = A.nx, ny = A.ny, nz = A.nz, V = A.V;
    const int ix = j % nx, r = j / nx, iy = r % ny, iz = r / ny;
    const bool inx = ix < nx - 1, iny = iy < ny - 1, inz = iz < nz - 1;
    const float u0 = A.ubar[j];
    const float ux = (A.cx >= 0 && inx) ? A.ubar[j + 1] : u0;
    const float uy = (A.cy >= 0 && iny) ? A.ubar[j + nx] : u0;
    const float uz = (A.cz >= 0 && inz) ? A.ubar[j + nx * ny] : u0;
    const float q0 = A.cx >= 0 ? A.q[A.cx * V + j] : 0.0f;
    const float q1 = A.cy >= 0 ? A.q[A.cy * V + j] : 0.0f;
    const float q2 = A.cz >= 0 ? A.q[A.cz * V + j] : 0.0f;
    float o0, o1, o2;
    dual_point(A, sg, u0, ux, uy, uz, inx, iny, inz, q0, q1, q2, o0, o1, o2);
    if (A.cx >= 0) A.q[A.cx * V + j] = o0;
    if (A.cy >= 0) A.q[A.cy * V + j] = o1;
    if (A.cz >= 0) A.q[A.cz * V + j] = o2;
}

__global__ void __launch_bounds__(256) primal_point_kernel(const PdArgs A)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= A.V) return;
    const float tau = A.sc->tau[A.k], th = A.sc->theta[A.k];
    const int nx = A.nx, ny = A.ny, nz = A.nz, V = A.V;
    const int ix = j % nx, r = j / nx, iy = r % ny, iz = r / ny;
    float kt = 0.0f;
    if (A.cx >= 0) {
        if (ix < nx - 1) kt -= A.q[A.cx * V + j];
        if (ix >= 1) kt += A.q[A.cx * V + j - 1];
    }
    if (A.cy >= 0) {
        if (iy < ny - 1) kt -= A.q[A.cy * V + j];
        if (iy >= 1) kt += A.q[A.cy * V + j - nx];
    }
    if (A.cz >= 0) {
        if (iz < nz - 1) kt -= A.q[A.cz * V + j];
        if (iz >= 1) kt += A.q[A.cz * V + j - nx * ny];
    }
    float ub;
    A.u[j] = primal_point(tau, th, kt, A.u[j], A.w[j], A.z[j], ub);
    A.ubar[j] = ub;
}

int voxel_grid(int64_t V)
{
    const int64_t want = (V + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 8));
}

// The schedule from gam, then the inner iterations on (u, ubar, q) with z, w.
int run_pdhg(const lm_grid* g, const Ws& W, float* u, int iters, double knorm, cudaStream_t st)
{
    sched_kernel<<<1, 32, 0, st>>>(W.sc, iters, knorm);
    count_launch();
    PdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = g->n[0];
    a.ny = g->n[1];
    a.nz = g->n[2];
    int c = 0;
    a.cx = a.nx > 1 ? c++ : -1;
    a.cy = a.ny > 1 ? c++ : -1;
    a.cz = a.nz > 1 ? c++ : -1;
    a.V = (int)nvox(g);
    a.ubar = W.ubar;
    a.q = W.q;
    a.u = u;
    a.z = W.z;
    a.w = W.w;
    a.sc = W.sc;
    const bool quad = (a.nx & 3) == 0;
    const int blocks = quad ? (a.V / 4 + 255) / 256 : (a.V + 255) / 256;
    for (int k = 0; k < iters; ++k) {
        a.k = k;
        if (quad) {
            dual_quad_kernel<<<blocks, 256, 0, st>>>(a);
            primal_quad_kernel<<<blocks, 256, 0, st>>>(a);
        } else {
            dual_point_kernel<<<blocks, 256, 0, st>>>(a);
            primal_point_kernel<<<blocks, 256, 0, st>>>(a);
        }
    }
    count_launch(2 * (int64_t)iters);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int check_common(const lm_grid* grid, void* ws, size_t ws_bytes, int iters, double knorm)
{
    int rc = check_grid(grid);
    if (rc) return rc;
    LM_CHECK(ws != nullptr && ws_bytes >= ws_layout(grid, nullptr, nullptr), LM_ERR_NOMEM,
             "EM-TV needs %zu workspace bytes", ws_layout(grid, nullptr, nullptr));
    LM_CHECK(((uintptr_t)ws & 255) == 0, LM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    LM_CHECK(iters >= 0 && iters <= EMTV_MAX_ITERS, LM_ERR_INVALID_ARG, "pdhg_iters must be in [0, %d]",
             EMTV_MAX_ITERS);
    LM_CHECK(std::isfinite(knorm) && knorm > 0.0, LM_ERR_INVALID_ARG, "knorm must be positive");
    return LM_OK;
}

// Back-projection of c_e / (c_e J_e x + s_e) over events [e0, e1) into W.z
// (overwritten; scattered into the pair accumulators of both layouts like the
// LM-SPDHG data update, then folded into one image), then em_fold_kernel.
int em_step(const lm_scanner* sc, const lm_grid* grid, const Geo& G, const lm_events* ev, int64_t e0, int64_t e1,
            int n_subsets, const float* sens, float* x, float beta, const Ws& W, cudaStream_t st)
{
    const size_t V = (size_t)nvox(grid);
    const bool two_d = grid->n[2] == 1 && sc->n_rings == 1;  // single-ring scanner in the image plane
    const bool use_yf = grid->n[1] > 1;
    if (beta > 0.0f) LM_CUDA(cudaMemsetAsync(&W.sc->gam_nbits, 0, 4, st));
    if (e1 <= e0) LM_CUDA(cudaMemsetAsync(W.z, 0, V * 4, st));
    if (e1 > e0) {
        EvArgs a;
        std::memset(&a, 0, sizeof(a));
        a.G = G;
        a.x_std = x;
        a.det1 = ev->det1;
        a.det2 = ev->det2;
        a.tof = ev->tof;
        a.corr = ev->corr;
        a.contam = ev->contam;
        a.acc_std = W.pair_std;
        a.acc_pairs = 1;
        if (use_yf) {
            launch_transpose_to_yf(grid, x, W.x_yf, st);
            a.x_yf = W.x_yf;
            a.acc_yf = W.pair_yf;
        }
        a.e_begin = e0;
        a.e_end = e1;
        a.chunk = 32;
        a.queue = &W.sc->queue;
        a.done = &W.sc->done;
        a.tof_tab = G.tof_on ? W.tof_tab : nullptr;
        a.group = two_d ? 16 : 32;  // the widths the autotuner picks on the 2D and 3D frames
        a.stepmax = 2.0f * std::fmax(grid->h[0], std::fmax(grid->h[1], grid->h[2]));
        int rc = launch_events(EV_EM, two_d, a, ev_grid_g(EV_EM, two_d, a.group), st);
        LM_CHECK(rc == LM_OK, rc, "EM back-projection launch failed");
        launch_res_fold(grid, W.pair_std, W.pair_yf, W.z, nullptr, 0, 0, st);
    }
    const Axes ax = axes_of(grid);
    em_fold_kernel<<<voxel_grid((int64_t)V), 256, 0, st>>>(x, W.z, sens, W.w, W.ubar, W.q, std::max(1, ax.nd),
                                                          (int64_t)V, (float)n_subsets, beta, W.sc);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// Same checks as the projector's entry points.
int check_events_em(const lm_tof* tof, const lm_events* ev)
{
    LM_CHECK(ev != nullptr && ev->n >= 0, LM_ERR_INVALID_ARG, "events NULL or negative count");
    if (ev->n == 0) return LM_OK;
    LM_CHECK(ev->det1 && ev->det2, LM_ERR_INVALID_ARG, "event detector arrays are NULL");
    LM_CHECK(ev->contam != nullptr, LM_ERR_INVALID_ARG, "event contamination is NULL");
    LM_CHECK(tof->n_bins == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    return LM_OK;
}

}  // namespace

extern "C" {

size_t lm_emtv_workspace_bytes(const lm_grid* grid)
{
    if (check_grid(grid)) return 0;
    return ws_layout(grid, nullptr, nullptr);
}

int lm_emtv_em_step(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
                    int32_t n_subsets, const float* sens, const float* x, float* z, void* ws, size_t ws_bytes,
                    void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    rc = check_common(grid, ws, ws_bytes, 0, 1.0);
    if (rc) return rc;
    rc = check_events_em(tof, ev);
    if (rc) return rc;
    LM_CHECK(sens && x && z, LM_ERR_INVALID_ARG, "sens, x or z is NULL");
    LM_CHECK(n_subsets >= 1, LM_ERR_INVALID_ARG, "n_subsets must be >= 1");
    Ws W;
    ws_layout(grid, &W, ws);
    cudaStream_t st = S(stream);
    const size_t V = (size_t)nvox(grid);
    // work on a copy of x so that the fold (which writes x = z without a prior) leaves x untouched
    LM_CUDA(cudaMemcpyAsync(z, x, V * 4, cudaMemcpyDeviceToDevice, st));
    rc = em_prepare(grid, tof, W, st);
    if (rc) return rc;
    rc = em_step(sc, grid, G, ev, 0, ev->n, n_subsets, sens, z, 0.0f, W, st);
    if (rc) return rc;
    return LM_OK;
}

int lm_emtv_denoise(const lm_grid* grid, const float* z, const float* w, float* u, int32_t iters, double knorm,
                    void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    int rc = check_common(grid, ws, ws_bytes, iters, knorm);
    if (rc) return rc;
    LM_CHECK(z && w && u, LM_ERR_INVALID_ARG, "z, w or u is NULL");
    Ws W;
    ws_layout(grid, &W, ws);
    cudaStream_t st = S(stream);
    const size_t V = (size_t)nvox(grid);
    const Axes ax = axes_of(grid);
    LM_CUDA(cudaMemcpyAsync(W.z, z, V * 4, cudaMemcpyDeviceToDevice, st));
    LM_CUDA(cudaMemcpyAsync(W.w, w, V * 4, cudaMemcpyDeviceToDevice, st));
    LM_CUDA(cudaMemsetAsync(&W.sc->gam_nbits, 0, 4, st));
    denoise_init_kernel<<<voxel_grid((int64_t)V), 256, 0, st>>>(W.z, W.w, u, W.ubar, W.q, std::max(1, ax.nd),
                                                                (int64_t)V, W.sc);
    count_launch();
    LM_CUDA(cudaGetLastError());
    return run_pdhg(grid, W, u, iters, knorm, st);
}

int lm_emtv_epoch(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev_perm,
                  const int64_t* sub_off_host, int32_t n_subsets, const float* sens, float* x, float beta,
                  int32_t pdhg_iters, double knorm, void* ws, size_t ws_bytes, void* stream)
{
    clear_error();
    Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    rc = check_common(grid, ws, ws_bytes, pdhg_iters, knorm);
    if (rc) return rc;
    rc = check_events_em(tof, ev_perm);
    if (rc) return rc;
    LM_CHECK(sens && x, LM_ERR_INVALID_ARG, "sens or x is NULL");
    LM_CHECK(n_subsets >= 1 && sub_off_host != nullptr, LM_ERR_INVALID_ARG, "bad subset split");
    LM_CHECK(beta >= 0.0f && std::isfinite(beta), LM_ERR_INVALID_ARG, "beta must be finite and >= 0");
    LM_CHECK(sub_off_host[0] == 0 && sub_off_host[n_subsets] == ev_perm->n, LM_ERR_INVALID_ARG,
             "subset offsets must span [0, n)");
    for (int i = 0; i < n_subsets; ++i)
        LM_CHECK(sub_off_host[i + 1] >= sub_off_host[i], LM_ERR_INVALID_ARG, "subset offsets must not decrease");
    Ws W;
    ws_layout(grid, &W, ws);
    cudaStream_t st = S(stream);
    rc = em_prepare(grid, tof, W, st);
    if (rc) return rc;
    for (int i = 0; i < n_subsets; ++i) {
        rc = em_step(sc, grid, G, ev_perm, sub_off_host[i], sub_off_host[i + 1], n_subsets, sens, x, beta, W, st);
        if (rc) return rc;
        if (beta > 0.0f) {
            rc = run_pdhg(grid, W, x, pdhg_iters, knorm, st);
            if (rc) return rc;
        }
    }
    return LM_OK;
}

}  // extern "C"
