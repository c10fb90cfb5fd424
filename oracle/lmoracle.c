/*
 * FP64 CPU oracle for listmode SPDHG (LM-SPDHG) with a TOF Joseph projector.
 *
 * TEST INFRASTRUCTURE.  This file is the slow, plain reference that the CUDA
 * library is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * Everything is computed in double precision, single threaded, in the order
 * the paper states it:
 *   - Eq. (1)      primal objective  sum_i (Px+s)_i - d_i log (Px+s)_i + beta R(Kx)
 *   - Eq. (proxD)  prox of the Poisson conjugate, with d_i replaced by the
 *                  event count mu_e (appendix: rescaled operator, d^LM = 1)
 *   - Eq. (yinit)  optimal dual initialisation y = 1 - d/(Px+s)
 *   - Eq. (lmop)   listmode operator (P^LM x)_e = (Px)_{i_e}
 *   - Alg. 2       LM-SPDHG loop; Alg. 1 (SPDHG on a sinogram) for the
 *                  equivalence check of the appendix
 *   - Eq. (lm_stepsizes) step sizes S_k, T_k; S_{n+1}, T_{n+1} of Sec. 1
 *   - Sec. "Numerical experiments": TV prior ||Kx||_{2,1}, prox of R^*, and the
 *                  directional TV prior (K = P grad with a structural field)
 *   - Eq. (1)      P with an image-space resolution model: P = A G (or_res_apply)
 *
 * The projector: the paper cites Joseph (1982) and a Gaussian TOF kernel but
 * prints no formula.  The reading implemented here:
 *   endpoints a = xtal[det1], b = xtal[det2] (float32 table values);
 *   principal axis k = argmax_j |fl32(b_j - a_j)| (ties -> lowest j);
 *   for every voxel plane i along k: lambda = (o_k + i h_k - a_k)/(b_k - a_k),
 *   p = a + lambda (b - a); bilinear interpolation over the two other axes
 *   with neighbours outside the grid contributing 0; sample weight
 *   step = h_k |b - a| / |b_k - a_k|;
 *   TOF position t = (lambda - 1/2)|b - a| (from the LOR centre toward det2),
 *   bin centre c_m = m * bin; bin-integrated Gaussian
 *   w_m(t) = 1/2 [erf((t - c_m + bin/2)/(sqrt2 sigma)) - erf((t - c_m - bin/2)/(sqrt2 sigma))],
 *   kept iff |t - c_m| <= n_sigma * sigma.
 *   J_e(x) = sum_i step * w_m(t_i) * interp(x, p_i); (P^LM x)_e = corr_e J_e(x).
 *   The detectors lie outside the image, so the infinite line and the
 *   detector-to-detector segment cross the same voxels.
 *
 *   - Alg. 3       listmode EM-TV (the warm start x0): subset EM step and
 *                  weighted TV denoising by accelerated primal-dual iterations
 *
 * parity pinned: adjoint, TOF sum, closed-form chords, brute force on tiny
 * grids, prox fixed points, TV adjoint and norm, LM == sinogram SPDHG; EM-TV:
 * the EM step as a scaled log-likelihood gradient step (finite differences),
 * the denoiser's closed form (two voxels), an independent dual solve,
 * optimality conditions, Chambolle-Pock's asymptotic and non-asymptotic
 * rate bounds (the latter fails without the extrapolation) and limits; the
 * iterate path at a fixed iteration count against the first ten iterates of
 * the two-voxel problem in 40-digit arithmetic (see the CPU tests).  The two
 * tolerance helpers at the end are pinned through the forward projector:
 * the TOF cut margin by moving the cut, the position sensitivity by finite
 * differences under a detector shift.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_rings, n_xtal;
    const float* xtal; /* [n_rings*n_xtal][3] */
} or_scanner;

typedef struct {
    int32_t n[3];
    float h[3];
    float origin[3];
} or_grid;

typedef struct {
    float sigma, bin, n_sigma;
    int32_t n_bins; /* odd; 0 = non-TOF */
} or_tof;

/* kernel mode of one projection */
enum { OR_NONTOF = 0, OR_TOFBIN = 1, OR_TOFSUM = 2 };

typedef void (*or_visit)(void* ctx, int64_t j, double w);

static double tof_bin_weight(double tau, const or_tof* tof)
{
    double sig = (double)tof->sigma, D = (double)tof->bin;
    if (fabs(tau) > (double)tof->n_sigma * sig) return 0.0;
    double s = sqrt(2.0) * sig;
    return 0.5 * (erf((tau + 0.5 * D) / s) - erf((tau - 0.5 * D) / s));
}

/* Visit every (voxel, weight) pair of the Joseph projection of one LOR. */
static void or_lor_visit(const or_scanner* sc, const or_grid* g, const or_tof* tof, int32_t d1,
                         int32_t d2, int32_t m, int mode, or_visit f, void* ctx)
{
    double a[3], b[3], d[3], o[3], h[3];
    float df[3];
    int j;
    for (j = 0; j < 3; ++j) {
        a[j] = (double)sc->xtal[3 * (int64_t)d1 + j];
        b[j] = (double)sc->xtal[3 * (int64_t)d2 + j];
        d[j] = b[j] - a[j]; /* exact: difference of two float32 values */
        df[j] = (float)d[j];
        o[j] = (double)g->origin[j];
        h[j] = (double)g->h[j];
    }
    int k = 0;
    if (fabsf(df[1]) > fabsf(df[k])) k = 1;
    if (fabsf(df[2]) > fabsf(df[k])) k = 2;
    if (d[k] == 0.0) return;
    int s1 = (k + 1) % 3, s2 = (k + 2) % 3;
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double step = h[k] * L / fabs(d[k]);
    for (int i = 0; i < g->n[k]; ++i) {
        double qk = o[k] + i * h[k];
        double lam = (qk - a[k]) / d[k];
        double p[3];
        for (j = 0; j < 3; ++j) p[j] = a[j] + lam * d[j];
        double t = (lam - 0.5) * L;
        double wt = 1.0;
        if (mode == OR_TOFBIN) {
            wt = tof_bin_weight(t - (double)m * (double)tof->bin, tof);
        } else if (mode == OR_TOFSUM) {
            int M = (tof->n_bins - 1) / 2;
            wt = 0.0;
            for (int mm = -M; mm <= M; ++mm) wt += tof_bin_weight(t - (double)mm * (double)tof->bin, tof);
        }
        if (wt == 0.0) continue;
        double u1 = (p[s1] - o[s1]) / h[s1];
        double u2 = (p[s2] - o[s2]) / h[s2];
        double fl1 = floor(u1), fl2 = floor(u2);
        int64_t i1 = (int64_t)fl1, i2 = (int64_t)fl2;
        double f1 = u1 - fl1, f2 = u2 - fl2;
        for (int da = 0; da < 2; ++da) {
            int64_t j1 = i1 + da;
            if (j1 < 0 || j1 >= g->n[s1]) continue;
            double w1 = da ? f1 : 1.0 - f1;
            for (int db = 0; db < 2; ++db) {
                int64_t j2 = i2 + db;
                if (j2 < 0 || j2 >= g->n[s2]) continue;
                double w2 = db ? f2 : 1.0 - f2;
                int64_t idx[3];
                idx[k] = i;
                idx[s1] = j1;
                idx[s2] = j2;
                int64_t vox = (idx[2] * g->n[1] + idx[1]) * g->n[0] + idx[0];
                f(ctx, vox, step * wt * w1 * w2);
            }
        }
    }
}

typedef struct {
    const float* xf;
    const double* xd;
    double acc;
} fwd_ctx;

static void fwd_visit(void* c, int64_t j, double w)
{
    fwd_ctx* q = (fwd_ctx*)c;
    q->acc += w * (q->xf ? (double)q->xf[j] : q->xd[j]);
}

typedef struct {
    double* img;
    double v;
} back_ctx;

static void back_visit(void* c, int64_t j, double w)
{
    back_ctx* q = (back_ctx*)c;
    q->img[j] += w * q->v;
}

static void ones_visit(void* c, int64_t j, double w)
{
    (void)j;
    ((fwd_ctx*)c)->acc += w;
}

static int ev_mode(const or_tof* tof) { return tof->n_bins > 0 ? OR_TOFBIN : OR_NONTOF; }

/* (P^LM x)_e = corr_e J_e(x) for float32 x (Eq. lmop). corr may be NULL (=1). */
void or_fwd(const or_scanner* sc, const or_grid* g, const or_tof* tof, const int32_t* det1,
            const int32_t* det2, const int16_t* tbin, const float* corr, int64_t n, const float* x,
            double* out)
{
    for (int64_t e = 0; e < n; ++e) {
        fwd_ctx c = {x, NULL, 0.0};
        or_lor_visit(sc, g, tof, det1[e], det2[e], tbin[e], ev_mode(tof), fwd_visit, &c);
        out[e] = c.acc * (corr ? (double)corr[e] : 1.0);
    }
}

/* img += (P^LM)^T v, i.e. img += sum_e corr_e J_e^T v_e. */
void or_back(const or_scanner* sc, const or_grid* g, const or_tof* tof, const int32_t* det1,
             const int32_t* det2, const int16_t* tbin, const float* corr, int64_t n,
             const double* v, double* img)
{
    for (int64_t e = 0; e < n; ++e) {
        back_ctx c = {img, v[e] * (corr ? (double)corr[e] : 1.0)};
        or_lor_visit(sc, g, tof, det1[e], det2[e], tbin[e], ev_mode(tof), back_visit, &c);
    }
}

/* Non-TOF projection of single LORs (used for chord pins). */
void or_fwd_nontof(const or_scanner* sc, const or_grid* g, const int32_t* det1,
                   const int32_t* det2, int64_t n, const double* x, double* out)
{
    or_tof t = {1.0f, 1.0f, 3.0f, 0};
    for (int64_t e = 0; e < n; ++e) {
        fwd_ctx c = {NULL, x, 0.0};
        or_lor_visit(sc, g, &t, det1[e], det2[e], 0, OR_NONTOF, fwd_visit, &c);
        out[e] = c.acc;
    }
}

/* Sum over all TOF bins of one LOR, by explicit per-bin projection (TOF-sum pin). */
double or_lor_tofsum_fwd(const or_scanner* sc, const or_grid* g, const or_tof* tof, int32_t d1,
                         int32_t d2, const double* x)
{
    int M = (tof->n_bins - 1) / 2;
    double s = 0.0;
    for (int m = -M; m <= M; ++m) {
        fwd_ctx c = {NULL, x, 0.0};
        or_lor_visit(sc, g, tof, d1, d2, m, OR_TOFBIN, fwd_visit, &c);
        s += c.acc;
    }
    return s;
}

/* Canonical LOR l -> (det1, det2); see the scanner description in the tests. */
static void lor_dets(const or_scanner* sc, int64_t l, int32_t* d1, int32_t* d2)
{
    int64_t nr = sc->n_rings, n = sc->n_xtal;
    int64_t rb = l % nr;
    int64_t ra = (l / nr) % nr;
    int64_t q = l / (nr * nr);
    int64_t base = n * ((n - 1) / 2);
    int64_t c1, c2;
    if (q < base) {
        c1 = q % n;
        c2 = (c1 + 1 + q / n) % n;
    } else {
        c1 = q - base;
        c2 = c1 + n / 2;
    }
    *d1 = (int32_t)(ra * n + c1);
    *d2 = (int32_t)(rb * n + c2);
}

int64_t or_n_lor(const or_scanner* sc)
{
    return (int64_t)sc->n_xtal * (sc->n_xtal - 1) / 2 * sc->n_rings * sc->n_rings;
}

void or_lor_dets(const or_scanner* sc, int64_t l, int32_t* d1, int32_t* d2) { lor_dets(sc, l, d1, d2); }

/* Sensitivity image P^T 1: every canonical LOR, every TOF bin (plain sum over
 * bins), times the LOR factor (NULL = 1).  Sec. "Listmode SPDHG": "pre-compute
 * the sensitivity image and store it". */
void or_sens(const or_scanner* sc, const or_grid* g, const or_tof* tof, const float* lor_factor,
             double* sens)
{
    int64_t nl = or_n_lor(sc);
    int mode = tof->n_bins > 0 ? OR_TOFSUM : OR_NONTOF;
    for (int64_t l = 0; l < nl; ++l) {
        int32_t d1, d2;
        lor_dets(sc, l, &d1, &d2);
        back_ctx c = {sens, lor_factor ? (double)lor_factor[l] : 1.0};
        or_lor_visit(sc, g, tof, d1, d2, 0, mode, back_visit, &c);
    }
}

/* ------------------------------------------------------------------------
 * Event counts mu_e (Alg. 2 "Calculate event counts"; footnote: a data bin
 * is the geometrical LOR together with the TOF bin).  The bin of an event is
 * its unordered detector pair with the TOF bin signed toward the larger
 * detector id.  Counting is over the whole list.
 * ------------------------------------------------------------------------ */
typedef struct {
    int32_t lo, hi, t;
    int64_t e;
} ev_key;

static int key_cmp(const void* A, const void* B)
{
    const ev_key* a = (const ev_key*)A;
    const ev_key* b = (const ev_key*)B;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    if (a->t != b->t) return a->t < b->t ? -1 : 1;
    return 0;
}

void or_event_counts(const int32_t* det1, const int32_t* det2, const int16_t* tbin, int64_t n,
                     int32_t* mu)
{
    ev_key* k = (ev_key*)malloc(sizeof(ev_key) * (size_t)(n > 0 ? n : 1));
    for (int64_t e = 0; e < n; ++e) {
        int swap = det1[e] > det2[e];
        k[e].lo = swap ? det2[e] : det1[e];
        k[e].hi = swap ? det1[e] : det2[e];
        k[e].t = swap ? -(int32_t)tbin[e] : (int32_t)tbin[e];
        k[e].e = e;
    }
    qsort(k, (size_t)n, sizeof(ev_key), key_cmp);
    int64_t s = 0;
    while (s < n) {
        int64_t t = s + 1;
        while (t < n && key_cmp(&k[s], &k[t]) == 0) ++t;
        for (int64_t r = s; r < t; ++r) mu[k[r].e] = (int32_t)(t - s);
        s = t;
    }
    free(k);
}

/* ------------------------------------------------------------------------
 * TV prior (Sec. "Numerical experiments"): K = finite forward differences
 * with unit spacing, last difference 0 (Neumann); one component per axis
 * with more than one voxel, in axis order x, y, z.  R = mixed L2-L1 norm.
 * ------------------------------------------------------------------------ */
static int tv_axes(const or_grid* g, int* ax)
{
    int nd = 0;
    for (int d = 0; d < 3; ++d)
        if (g->n[d] > 1) ax[nd++] = d;
    return nd;
}

int or_tv_ndim(const or_grid* g)
{
    int ax[3];
    return tv_axes(g, ax);
}

static int64_t stride_of(const or_grid* g, int d) { return d == 0 ? 1 : d == 1 ? g->n[0] : (int64_t)g->n[0] * g->n[1]; }

static int coord_of(const or_grid* g, int64_t j, int d)
{
    if (d == 0) return (int)(j % g->n[0]);
    if (d == 1) return (int)((j / g->n[0]) % g->n[1]);
    return (int)(j / ((int64_t)g->n[0] * g->n[1]));
}

/* out[c*V + j] = (Kx)_{j,c} */
void or_tv_grad(const or_grid* g, const double* x, double* out)
{
    int ax[3];
    int nd = tv_axes(g, ax);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    for (int c = 0; c < nd; ++c) {
        int d = ax[c];
        int64_t st = stride_of(g, d);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < V; ++j)
            out[c * V + j] = coord_of(g, j, d) < g->n[d] - 1 ? x[j + st] - x[j] : 0.0;
    }
}

/* out = K^T q (the adjoint of or_tv_grad); -div q. */
void or_tv_adj(const or_grid* g, const double* q, double* out)
{
    int ax[3];
    int nd = tv_axes(g, ax);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    for (int64_t j = 0; j < V; ++j) out[j] = 0.0;
    for (int c = 0; c < nd; ++c) {
        int d = ax[c];
        int64_t st = stride_of(g, d);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < V; ++j) {
            int cj = coord_of(g, j, d);
            if (cj < g->n[d] - 1) out[j] -= q[c * V + j];
            if (cj >= 1) out[j] += q[c * V + j - st];
        }
    }
}

/* w <- w / max(1, |w|/beta): beta * prox_{R^*}(w / beta), pointwise over
 * the per-voxel Euclidean norm of the components.  beta = 0 gives w = 0. */
void or_tv_prox(const or_grid* g, double* w, double beta)
{
    int nd = or_tv_ndim(g);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) {
        double s = 0.0;
        for (int c = 0; c < nd; ++c) s += w[c * V + j] * w[c * V + j];
        double nrm = sqrt(s);
        for (int c = 0; c < nd; ++c) {
            if (beta <= 0.0)
                w[c * V + j] = 0.0;
            else
                w[c * V + j] = w[c * V + j] / fmax(1.0, nrm / beta);
        }
    }
}

/* ------------------------------------------------------------------------
 * Directional TV (Sec. "Numerical experiments", after Ehrhardt & Betcke 2016):
 * only the part of the forward-difference vector perpendicular to the
 * gradient of a structural image counts,
 *   (K x)_j = P_j (grad x)_j,   P_j = I - xi_j xi_j^T,
 * with the per-voxel vector field xi ([nd][V], |xi_j| <= 1; NULL = TV).
 * K^T q = grad^T (P q) (P_j is symmetric).  The field of a structural image
 * v is xi_j = (grad v)_j / sqrt(|(grad v)_j|^2 + eta^2) (0 where both vanish);
 * eta = 0 makes P_j the orthogonal projection perpendicular to (grad v)_j.
 * ------------------------------------------------------------------------ */
static void dtv_project(const or_grid* g, const double* xi, double* q)
{
    int nd = or_tv_ndim(g);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) {
        double s = 0.0;
        for (int c = 0; c < nd; ++c) s += xi[c * V + j] * q[c * V + j];
        for (int c = 0; c < nd; ++c) q[c * V + j] -= xi[c * V + j] * s;
    }
}

void or_dtv_grad(const or_grid* g, const double* xi, const double* x, double* out)
{
    or_tv_grad(g, x, out);
    if (xi) dtv_project(g, xi, out);
}

void or_dtv_adj(const or_grid* g, const double* xi, const double* q, double* out)
{
    if (!xi) {
        or_tv_adj(g, q, out);
        return;
    }
    int nd = or_tv_ndim(g);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    double* t = (double*)malloc(sizeof(double) * V * (nd > 0 ? nd : 1));
    memcpy(t, q, sizeof(double) * V * nd);
    dtv_project(g, xi, t);
    or_tv_adj(g, t, out);
    free(t);
}

void or_dtv_xi(const or_grid* g, const double* v, double eta, double* xi)
{
    int nd = or_tv_ndim(g);
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    or_tv_grad(g, v, xi);
    for (int64_t j = 0; j < V; ++j) {
        double s = eta * eta;
        for (int c = 0; c < nd; ++c) s += xi[c * V + j] * xi[c * V + j];
        double r = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        for (int c = 0; c < nd; ++c) xi[c * V + j] *= r;
    }
}

/* ------------------------------------------------------------------------
 * Image-space resolution model.  Eq. (1)'s P includes the scanner's limited
 * spatial resolution; the paper gives no kernel.  Reading: P = A G with A the
 * TOF Joseph projector and G a separable Gaussian blur of full width at half
 * maximum fwhm (mm) on every axis with n_d > 1: sigma_d = fwhm / (2 sqrt(2 ln 2))
 * / h_d voxels, taps k = -r..r with r = floor(3 sigma_d + 1/2) (at most
 * n_d - 1), weights exp(-k^2 / (2 sigma_d^2)) normalised to sum 1, and the
 * image mirrored about its outer faces (index -1 reads 0, index n reads
 * n - 1).  That G is symmetric and its rows sum to 1, so P^T = G A^T and
 * P 1 = A 1.  fwhm <= 0: G = identity.
 * ------------------------------------------------------------------------ */
void or_res_apply(const or_grid* g, double fwhm, const double* x, double* out)
{
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    memcpy(out, x, sizeof(double) * V);
    if (!(fwhm > 0.0)) return;
    double* tmp = (double*)malloc(sizeof(double) * V);
    for (int d = 0; d < 3; ++d) {
        const int n = g->n[d];
        if (n < 2) continue;
        const double sig = fwhm / (2.0 * sqrt(2.0 * log(2.0))) / (double)g->h[d];
        int r = (int)floor(3.0 * sig + 0.5);
        if (r > n - 1) r = n - 1;
        double* w = (double*)malloc(sizeof(double) * (2 * r + 1));
        double sum = 0.0;
        for (int k = -r; k <= r; ++k) {
            w[k + r] = exp(-(double)k * k / (2.0 * sig * sig));
            sum += w[k + r];
        }
        for (int k = 0; k <= 2 * r; ++k) w[k] /= sum;
        const int64_t st = stride_of(g, d);
        for (int64_t j = 0; j < V; ++j) {
            const int c = coord_of(g, j, d);
            double acc = 0.0;
            for (int k = -r; k <= r; ++k) {
                int m = c + k;
                if (m < 0) m = -m - 1;
                if (m >= n) m = 2 * n - m - 1;
                acc += w[k + r] * out[j + (int64_t)(m - c) * st];
            }
            tmp[j] = acc;
        }
        memcpy(out, tmp, sizeof(double) * V);
        free(w);
    }
    free(tmp);
}

/* ||K|| by power iteration on K^T K from the checkerboard (-1)^(ix+iy+iz);
 * returns sqrt of the last Rayleigh quotient <v, K^T K v>/<v, v>. */
double or_knorm_power(const or_grid* g, int iters)
{
    int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    int nd = or_tv_ndim(g);
    double* v = (double*)malloc(sizeof(double) * V);
    double* gr = (double*)malloc(sizeof(double) * V * (nd > 0 ? nd : 1));
    double* u = (double*)malloc(sizeof(double) * V);
    for (int64_t j = 0; j < V; ++j) {
        int s = coord_of(g, j, 0) + coord_of(g, j, 1) + coord_of(g, j, 2);
        v[j] = (s & 1) ? -1.0 : 1.0;
    }
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        or_tv_grad(g, v, gr);
        or_tv_adj(g, gr, u);
        double vu = 0.0, vv = 0.0, uu = 0.0;
        for (int64_t j = 0; j < V; ++j) {
            vu += v[j] * u[j];
            vv += v[j] * v[j];
            uu += u[j] * u[j];
        }
        lam = vu / vv;
        double nu = sqrt(uu);
        if (nu == 0.0) break;
        for (int64_t j = 0; j < V; ++j) v[j] = u[j] / nu;
    }
    free(v);
    free(gr);
    free(u);
    return sqrt(lam);
}

/* ------------------------------------------------------------------------
 * Proximal map of the Poisson conjugate D^*(.; d) with step S (Eq. proxD):
 *   prox(a) = 1/2 (a + 1 - sqrt((a - 1)^2 + 4 S d)).
 * In the listmode algorithm d -> 1 and S -> mu_e S_e (appendix).
 * ------------------------------------------------------------------------ */
double or_prox_dstar(double a, double S, double d)
{
    return 0.5 * (a + 1.0 - sqrt((a - 1.0) * (a - 1.0) + 4.0 * S * d));
}

/* ------------------------------------------------------------------------
 * LM-SPDHG (Alg. 2).  State arrays are owned by the caller (numpy).
 * Event e belongs to subset e mod n (Sec. "Listmode SPDHG": every n-th event
 * goes to the n-th sub list).  Probabilities p_k = 1/(2n), p_{n+1} = 1/2.
 * ------------------------------------------------------------------------ */
typedef struct {
    const or_scanner* sc;
    const or_grid* g;
    const or_tof* tof;
    const int32_t *det1, *det2;
    const int16_t* tbin;
    const float *corr, *contam;
    const int32_t* mu;
    int64_t n_ev;
    int32_t n_subsets;
    double beta, gamma, rho, knorm;
    const double* xi; /* DTV field [nd][V]; NULL = TV */
    double res_fwhm;  /* resolution model G (mm, <= 0: none): P = A G */
} or_lm_problem;

typedef struct {
    double *x, *z, *zbar, *w, *y, *T;
} or_lm_state;

static double ev_fwd(const or_lm_problem* P, int64_t e, const double* x)
{
    fwd_ctx c = {NULL, x, 0.0};
    or_lor_visit(P->sc, P->g, P->tof, P->det1[e], P->det2[e], P->tbin[e], ev_mode(P->tof), fwd_visit, &c);
    return c.acc * (double)P->corr[e];
}

static double ev_fwd_ones(const or_lm_problem* P, int64_t e)
{
    fwd_ctx c = {NULL, NULL, 0.0};
    or_lor_visit(P->sc, P->g, P->tof, P->det1[e], P->det2[e], P->tbin[e], ev_mode(P->tof), ones_visit, &c);
    return c.acc * (double)P->corr[e];
}

static void ev_back(const or_lm_problem* P, int64_t e, double v, double* img)
{
    back_ctx c = {img, v * (double)P->corr[e]};
    or_lor_visit(P->sc, P->g, P->tof, P->det1[e], P->det2[e], P->tbin[e], ev_mode(P->tof), back_visit, &c);
}

/* The image the projector A reads: G x with the resolution model (a new
 * array in *buf), x itself without (*buf = NULL). */
static const double* res_in(const or_lm_problem* P, const double* x, double** buf)
{
    *buf = NULL;
    if (!(P->res_fwhm > 0.0)) return x;
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    *buf = (double*)malloc(sizeof(double) * V);
    or_res_apply(P->g, P->res_fwhm, x, *buf);
    return *buf;
}

/* img += G b (the transpose of the resolution model after a back-projection b). */
static void res_add(const or_lm_problem* P, const double* b, double* img)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    double* t = (double*)malloc(sizeof(double) * V);
    or_res_apply(P->g, P->res_fwhm, b, t);
    for (int64_t j = 0; j < V; ++j) img[j] += t[j];
    free(t);
}

/* (P^LM 1)_e = corr_e J_e(G 1) */
static double ev_fwd_one_img(const or_lm_problem* P, int64_t e, const double* g1)
{
    return g1 ? ev_fwd(P, e, g1) : ev_fwd_ones(P, e);
}

/* The event loops of Alg. 2 (the initialisation over every event, a data
 * update over the events e = e0, e0 + de, ...): each event's dual step is
 * its own, and its back-projection is added into img.  In the plain build
 * the events run in list order.  Built with OpenMP (the timing baseline on
 * all host cores), every thread adds into its own FP64 image, and those are
 * added into img in thread order after the loop. */
enum { STEP_INIT = 0, STEP_DATA = 1 };

static double event_step(const or_lm_problem* P, or_lm_state* S, int64_t e, int kind, const double* gx,
                         const double* g1)
{
    double mu = (double)P->mu[e];
    if (kind == STEP_INIT) {
        double u = ev_fwd(P, e, gx) + (double)P->contam[e];
        S->y[e] = 1.0 - mu / u;                                 /* Eq. (yinit) */
        return (S->y[e] - 1.0) / mu;
    }
    double p1 = ev_fwd_one_img(P, e, g1);
    double Se = p1 > 0.0 ? P->gamma * P->rho / p1 : 0.0;       /* S_k = gamma rho / P^LM_{N_k} 1 */
    double a = S->y[e] + Se * (ev_fwd(P, e, gx) + (double)P->contam[e]);
    double yp = or_prox_dstar(a, mu * Se, 1.0);
    double v = (yp - S->y[e]) / mu;
    S->y[e] = yp;
    return v;
}

static void event_pass(const or_lm_problem* P, or_lm_state* S, int64_t e0, int64_t de, int kind, const double* gx,
                       const double* g1, double* img)
{
#ifdef _OPENMP
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nt = omp_get_max_threads();
    double* part = (double*)calloc((size_t)nt * V, sizeof(double));
#pragma omp parallel
    {
        double* mine = part + (size_t)omp_get_thread_num() * V;
#pragma omp for schedule(dynamic, 64)
        for (int64_t e = e0; e < P->n_ev; e += de) ev_back(P, e, event_step(P, S, e, kind, gx, g1), mine);
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j)
        for (int t = 0; t < nt; ++t) img[j] += part[(size_t)t * V + j];
    free(part);
#else
    for (int64_t e = e0; e < P->n_ev; e += de) ev_back(P, e, event_step(P, S, e, kind, gx, g1), img);
#endif
}


/* Initialisation of Alg. 2 (duals, z, step sizes) plus the first primal step's inputs:
 *   y_e = 1 - mu_e / ((P^LM x0)_e + s_e)                    (Eq. yinit)
 *   z = zbar = P^T 1 + (P^LM)^T ((y - 1)/mu) + K^T w, w = 0
 *     (the sign reading: the first part equals P^T applied to a sinogram that
 *      is 1 on empty bins and Eq. yinit elsewhere)
 *   T_j = min_k T_k = (rho/gamma) min( p_k n / sens_j , p_{n+1} / ||K|| )  (Eq. lm_stepsizes)
 */
void or_lm_init(const or_lm_problem* P, const float* x0, const double* sens, or_lm_state* S)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    double* x0d = S->x;
    for (int64_t j = 0; j < V; ++j) x0d[j] = (double)x0[j];
    for (int64_t j = 0; j < V; ++j) S->z[j] = sens[j];
    double* gbuf;
    const double* gx = res_in(P, x0d, &gbuf);
    double* bz = gbuf ? (double*)calloc(V, sizeof(double)) : S->z;
    event_pass(P, S, 0, 1, STEP_INIT, gx, NULL, bz);  /* y, and (P^LM)^T((y - 1)/mu) into bz */
    if (gbuf) {
        res_add(P, bz, S->z);
        free(bz);
        free(gbuf);
    }
    for (int64_t j = 0; j < (int64_t)nd * V; ++j) S->w[j] = 0.0;
    for (int64_t j = 0; j < V; ++j) S->zbar[j] = S->z[j];
    double n = (double)P->n_subsets;
    double p_data = 1.0 / (2.0 * n), p_prior = 0.5;
    for (int64_t j = 0; j < V; ++j) {
        double t_prior = P->rho * p_prior / (P->gamma * P->knorm);
        double t_data = sens[j] > 0.0 ? P->rho * p_data / (P->gamma * sens[j] / n) : INFINITY;
        S->T[j] = t_data < t_prior ? t_data : t_prior;
    }
}

/* One iteration of the Alg. 2 loop with selection i (0..n-1 data subset,
 * n = prior).  dz is caller scratch of V doubles, gw of nd*V doubles. */
void or_lm_update(const or_lm_problem* P, or_lm_state* S, int32_t i, double* dz, double* gw)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    double n = (double)P->n_subsets;
    /* x <- proj_{>=0}(x - T zbar) */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) {
        double v = S->x[j] - S->T[j] * S->zbar[j];
        S->x[j] = v > 0.0 ? v : 0.0;
    }
    for (int64_t j = 0; j < V; ++j) dz[j] = 0.0;
    double p_i;
    if (i < P->n_subsets) {
        p_i = 1.0 / (2.0 * n);
        double *gbuf, *g1 = NULL;
        const double* gx = res_in(P, S->x, &gbuf);
        if (gbuf) {
            double* ones = (double*)malloc(sizeof(double) * V);
            for (int64_t j = 0; j < V; ++j) ones[j] = 1.0;
            g1 = (double*)malloc(sizeof(double) * V);
            or_res_apply(P->g, P->res_fwhm, ones, g1);
            free(ones);
        }
        double* bz = gbuf ? (double*)calloc(V, sizeof(double)) : dz;
        /* subset i: every n-th event from i; y+ = prox (Eq. proxD), dz += P^T (y+ - y)/mu */
        event_pass(P, S, i, P->n_subsets, STEP_DATA, gx, g1, bz);
        if (gbuf) {
            res_add(P, bz, dz);
            free(bz);
            free(gbuf);
            free(g1);
        }
    } else {
        p_i = 0.5;
        double Sp = P->gamma * P->rho / P->knorm; /* S_{n+1} */
        or_dtv_grad(P->g, P->xi, S->x, gw);
        for (int64_t j = 0; j < (int64_t)nd * V; ++j) gw[j] = S->w[j] + Sp * gw[j];
        or_tv_prox(P->g, gw, P->beta);                 /* gw = w^+ */
        for (int64_t j = 0; j < (int64_t)nd * V; ++j) {
            double t = gw[j];
            gw[j] = t - S->w[j];                       /* w^+ - w */
            S->w[j] = t;
        }
        or_dtv_adj(P->g, P->xi, gw, dz);               /* dz = K^T (w^+ - w) */
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) {
        S->z[j] += dz[j];
        S->zbar[j] = S->z[j] + dz[j] / p_i;
    }
}

/* Objective of Eq. (1) in listmode form without the constant sum of s over
 * all bins:  <P^T 1, x> - sum_e log((P^LM x)_e + s_e) + beta ||Kx||_{2,1}. */
double or_lm_objective(const or_lm_problem* P, const double* x, const double* sens)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    double c = 0.0;
    for (int64_t j = 0; j < V; ++j) c += sens[j] * x[j];
    double* gbuf;
    const double* gx = res_in(P, x, &gbuf);
    for (int64_t e = 0; e < P->n_ev; ++e) c -= log(ev_fwd(P, e, gx) + (double)P->contam[e]);
    free(gbuf);
    if (P->beta > 0.0) {
        double* gr = (double*)malloc(sizeof(double) * V * (nd > 0 ? nd : 1));
        or_dtv_grad(P->g, P->xi, x, gr);
        double r = 0.0;
        for (int64_t j = 0; j < V; ++j) {
            double s = 0.0;
            for (int cc = 0; cc < nd; ++cc) s += gr[cc * V + j] * gr[cc * V + j];
            r += sqrt(s);
        }
        free(gr);
        c += P->beta * r;
    }
    return c;
}

/* ------------------------------------------------------------------------
 * Listmode EM-TV (Alg. 3), the initialisation of x0 used in the paper's
 * experiments (one pass over the n subsets, Sec. "Numerical experiments").
 * Per subset i:
 *   z = x n / g * (P^LM_{N_i})^T (1 / (P^LM_{N_i} x + s_{N_i}))  (subset EM step;
 *       the printed step has no x inside P^LM_{N_i}: read as the current x)
 *   w = g / (beta x)
 *   x = argmin_{u >= 0} sum_j w_j/2 (u_j - z_j)^2 + ||K u||_{2,1}
 * The last problem is solved by the accelerated primal-dual algorithm of
 * Chambolle & Pock (2011, their Alg. 2), which the paper names, with
 * G(u) = sum_j w_j/2 (u_j - z_j)^2 + i_{u >= 0} (uniformly convex with modulus
 * gam = min_j w_j over the free voxels) and F^* the indicator of the unit
 * 2-norm balls.  Readings (the paper gives no parameters): voxels with
 * x_j = 0 or g_j = 0 are held at 0; u_0 = ubar_0 = z, q_0 = 0,
 * tau_0 = sigma_0 = 0.99 / ||K||; per iteration
 *   q <- proj(q + sigma K ubar);  u+ = prox_{tau G}(u - tau K^T q);
 *   theta = 1/sqrt(1 + 2 gam tau);  tau <- theta tau;  sigma <- sigma/theta;
 *   ubar = u+ + theta (u+ - u).
 * ------------------------------------------------------------------------ */

/* Subset EM step: z_j = x_j n / g_j * sum_{e in N_i} c_e J_e^T / (c_e J_e x + s_e)
 * (z_j = 0 where g_j = 0).  Event e belongs to subset e mod n. */
void or_emtv_em_step(const or_lm_problem* P, const double* sens, const double* x, int32_t i, double* z)
{
    const int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    for (int64_t j = 0; j < V; ++j) z[j] = 0.0;
    double* gbuf;
    const double* gx = res_in(P, x, &gbuf);
    double* bz = gbuf ? (double*)calloc(V, sizeof(double)) : z;
    for (int64_t e = i; e < P->n_ev; e += P->n_subsets) {
        const double u = ev_fwd(P, e, gx) + (double)P->contam[e];
        ev_back(P, e, 1.0 / u, bz);
    }
    if (gbuf) {
        res_add(P, bz, z);
        free(bz);
        free(gbuf);
    }
    for (int64_t j = 0; j < V; ++j) z[j] = sens[j] > 0.0 ? x[j] * (double)P->n_subsets / sens[j] * z[j] : 0.0;
}

/* Weighted TV denoising by the accelerated primal-dual algorithm (see
 * above).  free_[j] = 0 holds u_j at 0.  q: dual variable (ndim*V), output. */
void or_emtv_denoise(const or_grid* g, const double* z, const double* w, const unsigned char* free_, int iters,
                     double knorm, double* u, double* q)
{
    const int64_t V = (int64_t)g->n[0] * g->n[1] * g->n[2];
    const int nd = or_tv_ndim(g) > 0 ? or_tv_ndim(g) : 1;
    double gam = INFINITY;
    for (int64_t j = 0; j < V; ++j)
        if (free_[j] && w[j] < gam) gam = w[j];
    if (!(gam < INFINITY)) gam = 0.0;
    double* ubar = (double*)malloc(sizeof(double) * V);
    double* kt = (double*)malloc(sizeof(double) * V);
    double* gr = (double*)malloc(sizeof(double) * nd * V);
    for (int64_t j = 0; j < V; ++j) u[j] = ubar[j] = free_[j] ? z[j] : 0.0;
    for (int64_t j = 0; j < (int64_t)nd * V; ++j) q[j] = 0.0;
    double tau = 0.99 / knorm, sigma = 0.99 / knorm;
    for (int it = 0; it < iters; ++it) {
        or_tv_grad(g, ubar, gr);
        for (int64_t j = 0; j < (int64_t)nd * V; ++j) q[j] += sigma * gr[j];
        or_tv_prox(g, q, 1.0); /* projection onto the unit balls */
        or_tv_adj(g, q, kt);
        const double theta = 1.0 / sqrt(1.0 + 2.0 * gam * tau);
        for (int64_t j = 0; j < V; ++j) {
            double un = 0.0;
            if (free_[j]) {
                const double v = u[j] - tau * kt[j];
                un = fmax(0.0, (v + tau * w[j] * z[j]) / (1.0 + tau * w[j]));
            }
            ubar[j] = un + theta * (un - u[j]);
            u[j] = un;
        }
        tau *= theta;
        sigma /= theta;
    }
    free(ubar);
    free(kt);
    free(gr);
}

/* One EM-TV pass over the subsets 0..n-1 in order; x (in/out). */
void or_emtv_epoch(const or_lm_problem* P, const double* sens, double* x, int pdhg_iters)
{
    const int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    const int nd = or_tv_ndim(P->g) > 0 ? or_tv_ndim(P->g) : 1;
    double* z = (double*)malloc(sizeof(double) * V);
    double* w = (double*)malloc(sizeof(double) * V);
    double* q = (double*)malloc(sizeof(double) * nd * V);
    unsigned char* fr = (unsigned char*)malloc(V);
    for (int32_t i = 0; i < P->n_subsets; ++i) {
        or_emtv_em_step(P, sens, x, i, z);
        if (!(P->beta > 0.0)) {
            /* no prior: the weight is infinite and the update is the EM step */
            for (int64_t j = 0; j < V; ++j) x[j] = z[j];
            continue;
        }
        for (int64_t j = 0; j < V; ++j) {
            fr[j] = (x[j] > 0.0 && sens[j] > 0.0) ? 1 : 0;
            w[j] = fr[j] ? sens[j] / (P->beta * x[j]) : 0.0;
        }
        or_emtv_denoise(P->g, z, w, fr, pdhg_iters, P->knorm, x, q);
    }
    free(z);
    free(w);
    free(q);
    free(fr);
}

/* ------------------------------------------------------------------------
 * Sinogram SPDHG (Alg. 1) over every (LOR, TOF bin) of the scanner, with the
 * memory-efficient initialisation of Sec. "Memory-efficient SPDHG": y = 1 on
 * empty bins and Eq. (yinit) elsewhere; z = P^T y.  Bins are indexed
 * b = l * n_bins + (m + M).  Subset of bin b: sub[b] (caller-supplied).
 * Empty bins are processed like every other bin.  The primal step size uses
 * P^T 1 / n as in Eq. (lm_stepsizes) so that the dual parts can be compared
 * with the listmode algorithm update by update.
 * ------------------------------------------------------------------------ */
typedef struct {
    const or_scanner* sc;
    const or_grid* g;
    const or_tof* tof;
    const float* lor_factor; /* [n_lor] */
    const double* d;         /* counts [n_bins_total] */
    const double* s;         /* contamination [n_bins_total] */
    const int32_t* sub;      /* subset of each bin */
    int32_t n_subsets;
    double beta, gamma, rho, knorm;
    const double* xi; /* DTV field [nd][V]; NULL = TV */
} or_sino_problem;

static void bin_dets(const or_sino_problem* P, int64_t b, int32_t* d1, int32_t* d2, int32_t* m)
{
    int nb = P->tof->n_bins > 0 ? P->tof->n_bins : 1;
    int M = (nb - 1) / 2;
    lor_dets(P->sc, b / nb, d1, d2);
    *m = (int32_t)(b % nb) - M;
}

static double bin_fwd(const or_sino_problem* P, int64_t b, const double* x)
{
    int32_t d1, d2, m;
    bin_dets(P, b, &d1, &d2, &m);
    int nb = P->tof->n_bins > 0 ? P->tof->n_bins : 1;
    fwd_ctx c = {NULL, x, 0.0};
    or_lor_visit(P->sc, P->g, P->tof, d1, d2, m, ev_mode(P->tof), x ? fwd_visit : ones_visit, &c);
    return c.acc * (double)P->lor_factor[b / nb];
}

static void bin_back(const or_sino_problem* P, int64_t b, double v, double* img)
{
    int32_t d1, d2, m;
    bin_dets(P, b, &d1, &d2, &m);
    int nb = P->tof->n_bins > 0 ? P->tof->n_bins : 1;
    back_ctx c = {img, v * (double)P->lor_factor[b / nb]};
    or_lor_visit(P->sc, P->g, P->tof, d1, d2, m, ev_mode(P->tof), back_visit, &c);
}

int64_t or_sino_nbins(const or_sino_problem* P)
{
    int nb = P->tof->n_bins > 0 ? P->tof->n_bins : 1;
    return or_n_lor(P->sc) * nb;
}

/* y: [n_bins_total]; x (V) initialised from x0; z, zbar, w, T as in LM. */
void or_sino_init(const or_sino_problem* P, const float* x0, const double* sens, or_lm_state* S)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    int64_t NB = or_sino_nbins(P);
    for (int64_t j = 0; j < V; ++j) {
        S->x[j] = (double)x0[j];
        S->z[j] = 0.0;
    }
    for (int64_t b = 0; b < NB; ++b) {
        if (P->d[b] > 0.0)
            S->y[b] = 1.0 - P->d[b] / (bin_fwd(P, b, S->x) + P->s[b]);
        else
            S->y[b] = 1.0;
        bin_back(P, b, S->y[b], S->z); /* z = P^T y */
    }
    for (int64_t j = 0; j < (int64_t)nd * V; ++j) S->w[j] = 0.0;
    for (int64_t j = 0; j < V; ++j) S->zbar[j] = S->z[j];
    double n = (double)P->n_subsets;
    for (int64_t j = 0; j < V; ++j) {
        double t_prior = P->rho * 0.5 / (P->gamma * P->knorm);
        double t_data = sens[j] > 0.0 ? P->rho * (1.0 / (2.0 * n)) / (P->gamma * sens[j] / n) : INFINITY;
        S->T[j] = t_data < t_prior ? t_data : t_prior;
    }
}

void or_sino_update(const or_sino_problem* P, or_lm_state* S, int32_t i, double* dz, double* gw)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    int64_t NB = or_sino_nbins(P);
    double n = (double)P->n_subsets;
    for (int64_t j = 0; j < V; ++j) {
        double v = S->x[j] - S->T[j] * S->zbar[j];
        S->x[j] = v > 0.0 ? v : 0.0;
    }
    for (int64_t j = 0; j < V; ++j) dz[j] = 0.0;
    double p_i;
    if (i < P->n_subsets) {
        p_i = 1.0 / (2.0 * n);
        for (int64_t b = 0; b < NB; ++b) {
            if (P->sub[b] != i) continue;
            double p1 = bin_fwd(P, b, NULL);
            double Sb = p1 > 0.0 ? P->gamma * P->rho / p1 : 0.0;
            double a = S->y[b] + Sb * (bin_fwd(P, b, S->x) + P->s[b]);
            double yp = or_prox_dstar(a, Sb, P->d[b]);
            bin_back(P, b, yp - S->y[b], dz);
            S->y[b] = yp;
        }
    } else {
        p_i = 0.5;
        double Sp = P->gamma * P->rho / P->knorm;
        or_dtv_grad(P->g, P->xi, S->x, gw);
        for (int64_t j = 0; j < (int64_t)nd * V; ++j) gw[j] = S->w[j] + Sp * gw[j];
        or_tv_prox(P->g, gw, P->beta);
        for (int64_t j = 0; j < (int64_t)nd * V; ++j) {
            double t = gw[j];
            gw[j] = t - S->w[j];
            S->w[j] = t;
        }
        or_dtv_adj(P->g, P->xi, gw, dz);
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < V; ++j) {
        S->z[j] += dz[j];
        S->zbar[j] = S->z[j] + dz[j] / p_i;
    }
}

/* Eq. (1) over all bins: sum_b (Px+s)_b - d_b log(Px+s)_b + beta ||Kx||_{2,1}. */
double or_sino_objective(const or_sino_problem* P, const double* x)
{
    int64_t V = (int64_t)P->g->n[0] * P->g->n[1] * P->g->n[2];
    int nd = or_tv_ndim(P->g);
    int64_t NB = or_sino_nbins(P);
    double c = 0.0;
    for (int64_t b = 0; b < NB; ++b) {
        double u = bin_fwd(P, b, x) + P->s[b];
        c += u;
        if (P->d[b] > 0.0) c -= P->d[b] * log(u);
    }
    if (P->beta > 0.0) {
        double* gr = (double*)malloc(sizeof(double) * V * (nd > 0 ? nd : 1));
        or_dtv_grad(P->g, P->xi, x, gr);
        double r = 0.0;
        for (int64_t j = 0; j < V; ++j) {
            double s = 0.0;
            for (int cc = 0; cc < nd; ++cc) s += gr[cc * V + j] * gr[cc * V + j];
            r += sqrt(s);
        }
        free(gr);
        c += P->beta * r;
    }
    return c;
}

/* Distance (mm) from the TOF truncation edge of the event's sample nearest
 * to it: min over planes of | |t_i - c_m| - n_sigma sigma |, over samples
 * with at least one in-grid neighbour.  Events where it is tiny are
 * "boundary-ambiguous": float32 and FP64 may decide the cut differently. */
void or_tof_edge_distance(const or_scanner* sc, const or_grid* g, const or_tof* tof, const int32_t* det1,
                          const int32_t* det2, const int16_t* tbin, int64_t n, double* out)
{
    for (int64_t e = 0; e < n; ++e) {
        double a[3], b[3], d[3], o[3], h[3];
        float df[3];
        for (int j = 0; j < 3; ++j) {
            a[j] = (double)sc->xtal[3 * (int64_t)det1[e] + j];
            b[j] = (double)sc->xtal[3 * (int64_t)det2[e] + j];
            d[j] = b[j] - a[j];
            df[j] = (float)d[j];
            o[j] = (double)g->origin[j];
            h[j] = (double)g->h[j];
        }
        int k = 0;
        if (fabsf(df[1]) > fabsf(df[k])) k = 1;
        if (fabsf(df[2]) > fabsf(df[k])) k = 2;
        double best = INFINITY;
        if (d[k] != 0.0 && tof->n_bins > 0) {
            int s1 = (k + 1) % 3, s2 = (k + 2) % 3;
            double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double W = (double)tof->n_sigma * (double)tof->sigma;
            for (int i = 0; i < g->n[k]; ++i) {
                double lam = (o[k] + i * h[k] - a[k]) / d[k];
                double u1 = (a[s1] + lam * d[s1] - o[s1]) / h[s1];
                double u2 = (a[s2] + lam * d[s2] - o[s2]) / h[s2];
                if (u1 <= -1.0 || u1 >= g->n[s1] || u2 <= -1.0 || u2 >= g->n[s2]) continue;
                double tau = (lam - 0.5) * L - (double)tbin[e] * (double)tof->bin;
                double dist = fabs(fabs(tau) - W);
                if (dist < best) best = dist;
            }
        }
        out[e] = best;
    }
}

/* Sensitivity of (P^LM x)_e to a shift of the sample positions: per event
 * corr_e * sum over samples of step * w_tof * (|d interp/d u1| + |d interp/d u2|),
 * u in voxel units.  Times the float32 resolution of a voxel coordinate it
 * bounds the projection error that comes from representing positions in
 * float32 (used to state the per-event tolerance of the float32 projector). */
void or_fwd_position_sensitivity(const or_scanner* sc, const or_grid* g, const or_tof* tof,
                                 const int32_t* det1, const int32_t* det2, const int16_t* tbin,
                                 const float* corr, int64_t n, const float* x, double* out)
{
    for (int64_t e = 0; e < n; ++e) {
        double a[3], b[3], d[3], o[3], h[3];
        float df[3];
        for (int j = 0; j < 3; ++j) {
            a[j] = (double)sc->xtal[3 * (int64_t)det1[e] + j];
            b[j] = (double)sc->xtal[3 * (int64_t)det2[e] + j];
            d[j] = b[j] - a[j];
            df[j] = (float)d[j];
            o[j] = (double)g->origin[j];
            h[j] = (double)g->h[j];
        }
        int k = 0;
        if (fabsf(df[1]) > fabsf(df[k])) k = 1;
        if (fabsf(df[2]) > fabsf(df[k])) k = 2;
        double acc = 0.0;
        if (d[k] != 0.0) {
            int s1 = (k + 1) % 3, s2 = (k + 2) % 3;
            double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double step = h[k] * L / fabs(d[k]);
            for (int i = 0; i < g->n[k]; ++i) {
                double lam = (o[k] + i * h[k] - a[k]) / d[k];
                double wt = 1.0;
                if (tof->n_bins > 0) wt = tof_bin_weight((lam - 0.5) * L - (double)tbin[e] * (double)tof->bin, tof);
                if (wt == 0.0) continue;
                double u1 = (a[s1] + lam * d[s1] - o[s1]) / h[s1];
                double u2 = (a[s2] + lam * d[s2] - o[s2]) / h[s2];
                double fl1 = floor(u1), fl2 = floor(u2);
                int64_t i1 = (int64_t)fl1, i2 = (int64_t)fl2;
                double f1 = u1 - fl1, f2 = u2 - fl2;
                double v[2][2];
                for (int da = 0; da < 2; ++da)
                    for (int db = 0; db < 2; ++db) {
                        int64_t j1 = i1 + da, j2 = i2 + db;
                        v[da][db] = 0.0;
                        if (j1 < 0 || j1 >= g->n[s1] || j2 < 0 || j2 >= g->n[s2]) continue;
                        int64_t idx[3];
                        idx[k] = i;
                        idx[s1] = j1;
                        idx[s2] = j2;
                        v[da][db] = (double)x[(idx[2] * g->n[1] + idx[1]) * g->n[0] + idx[0]];
                    }
                double g1 = (1.0 - f2) * (v[1][0] - v[0][0]) + f2 * (v[1][1] - v[0][1]);
                double g2 = (1.0 - f1) * (v[0][1] - v[0][0]) + f1 * (v[1][1] - v[1][0]);
                /* an axis of one voxel has no in-plane position to round */
                acc += step * wt * ((g->n[s1] > 1 ? fabs(g1) : 0.0) + (g->n[s2] > 1 ? fabs(g2) : 0.0));
            }
        }
        out[e] = acc * (corr ? (double)corr[e] : 1.0);
    }
}

/* Threads of the OpenMP build (the timing baseline); the plain build has one. */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
