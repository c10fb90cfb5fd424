/*
 * lmspdhg.h - C ABI of liblmspdhg.so: listmode SPDHG (LM-SPDHG) for sparse
 * Poisson TOF PET data on one NVIDIA GB300 (sm_103a).
 *
 * Problem (Eq. 1 of Schramm & Holler, "Fast and memory-efficient
 * reconstruction of sparse Poisson data in listmode with non-smooth priors
 * with application to time-of-flight PET", arXiv 2201.05497):
 *     argmin_{x >= 0} sum_i (Px + s)_i - d_i log (Px + s)_i + beta ||Kx||_{2,1}
 * solved from a list of events by Alg. 2 (LM-SPDHG).  Each event is one count
 * (d^LM_e = 1, appendix); the event count mu_e carries the multiplicity of
 * its data bin.
 *
 * Conventions for every call:
 *  - Pointers named "device" are CUDA device pointers in the caller's
 *    context, owned by the caller (allocate them with any allocator, e.g.
 *    PyTorch).  The library never allocates device memory; calls that need
 *    scratch take a caller workspace whose size a *_workspace_bytes /
 *    *_state_bytes function reports.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are asynchronous on that stream unless documented as
 *    synchronous (those return host scalars or report data errors found on
 *    the device).
 *  - Every call returns an lm status; lm_last_error() gives a message for
 *    the calling thread's last failure.  Invalid host arguments are rejected
 *    before any launch.  Device-side data that would index out of range
 *    (detector ids, TOF bins) is skipped by the kernels, never dereferenced;
 *    lm_event_setup reports it as LM_ERR_OUT_OF_RANGE.
 *  - Images are float32, x fastest: voxel (ix, iy, iz) at (iz*ny + iy)*nx + ix.
 *    A 2D problem is a grid with n[2] = 1 and a one-ring scanner whose
 *    crystals lie in the plane of the voxel centres (z = origin[2]).
 *
 * Projector (the paper cites Joseph 1982 with a Gaussian TOF kernel and gives
 * no formula; this is the implemented definition):
 *   a = xtal[det1], b = xtal[det2]; principal axis k = argmax_j |b_j - a_j|
 *   (float32 differences, ties to the lowest j); one sample per voxel plane
 *   along k, at the line's crossing of the plane through the voxel centres;
 *   bilinear interpolation over the two other axes (neighbours outside the
 *   grid contribute 0); sample length h_k |b-a| / |b_k-a_k|.  TOF: t = signed
 *   distance of the sample from the LOR centre toward det2, bin centre m*bin,
 *   weight 1/2[erf((t-m bin+bin/2)/(sqrt2 sigma)) - erf((t-m bin-bin/2)/(sqrt2 sigma))]
 *   for |t - m bin| <= n_sigma sigma, else 0.
 *   (P^LM x)_e = corr_e * J_e(x)   (Eq. lmop; corr = attenuation x normalisation).
 */
#ifndef LMSPDHG_H
#define LMSPDHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LM_OK 0
#define LM_ERR_INVALID_ARG 1  /* bad host argument (NULL, size, geometry)     */
#define LM_ERR_OUT_OF_RANGE 2 /* detector id / TOF bin out of range, mu > 65535 */
#define LM_ERR_DOMAIN 3       /* x0 < 0, corr <= 0, contam <= 0, ...            */
#define LM_ERR_CUDA 4         /* a CUDA runtime call failed                     */
#define LM_ERR_TIMEOUT 5      /* a bounded device wait gave up                  */
#define LM_ERR_NOMEM 6        /* caller workspace / state buffer too small      */

/* Message of the calling thread's last failed call ("" if none). */
const char* lm_last_error(void);
/* Library ABI version (major*100 + minor). */
int lm_version(void);
/* sizeof of the descriptor structs as this library was built, in the order
 * lm_scanner, lm_grid, lm_tof, lm_events, lm_params, lm_server_config:
 * writes min(n, 6) values to out (host) and returns 6, so a binding can
 * check its own struct layouts before the first call. */
int lm_struct_sizes(size_t* out, int n);

/* ---- descriptors ------------------------------------------------------ */
/* Crystal centres, mm, float32 [n_rings*n_xtal][3] (device); crystal id =
 * ring*n_xtal + transaxial index.  n_rings*n_xtal < 2^27. */
typedef struct {
    int32_t n_rings, n_xtal;
    const float* xtal_xyz;
} lm_scanner;

/* Voxel grid: n = (nx, ny, nz), voxel size h (mm), centre of voxel 0 (mm).
 * nx*ny*nz < 2^31.  2D: nz = 1. */
typedef struct {
    int32_t n[3];
    float h[3];
    float origin[3];
} lm_grid;

/* TOF kernel: Gaussian sigma (mm) integrated over bins of width bin_mm,
 * truncated at n_sigma*sigma; n_bins odd (signed bins -(n_bins-1)/2 ..
 * (n_bins-1)/2), n_bins <= 255; n_bins = 0 is non-TOF. */
typedef struct {
    float sigma_mm, bin_mm, n_sigma;
    int32_t n_bins;
} lm_tof;

/* Listmode events, device arrays of length n: detector ids, signed TOF bin
 * (toward det2), multiplicative correction corr_e > 0 and expected
 * contamination s_e > 0 of the event's data bin (s^LM of Eq. lmop).
 * corr/contam may be NULL where a call says so. */
typedef struct {
    const int32_t* det1;
    const int32_t* det2;
    const int16_t* tof;
    const float* corr;
    const float* contam;
    int64_t n;
} lm_events;

/* ---- projector --------------------------------------------------------- */
/* p_e = (P^LM x)_e = corr_e J_e(x)  (Eq. lmop).  x: device image; p: device
 * float [ev->n].  corr NULL = 1.  ws (device, may be NULL) of at least
 * lm_fwd_workspace_bytes() lets y-principal events read a transposed copy
 * of x (faster gathers); results are the same either way up to rounding. */
size_t lm_fwd_workspace_bytes(const lm_grid* grid);
int lm_fwd(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const float* x,
           const lm_events* ev, float* p, void* ws, size_t ws_bytes, void* stream);

/* img += (P^LM)^T v = sum_e corr_e J_e^T v_e (adjoint of lm_fwd).  v: device
 * float [ev->n]; img: device image (accumulated into).  deterministic = 0:
 * float atomics (order of additions varies between runs); deterministic = 1:
 * every contribution is rounded to a 64-bit fixed-point grid whose step is
 * set from max|corr_e v_e| (at most 2^-62 of the largest possible voxel
 * sum), summed exactly with integer atomics and converted once, so the
 * result is bit-identical across runs and launch shapes.  ws: device
 * workspace of lm_back_workspace_bytes(grid, deterministic) bytes. */
size_t lm_back_workspace_bytes(const lm_grid* grid, int deterministic);
int lm_back(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
            const float* v, float* img, int deterministic, void* ws, size_t ws_bytes, void* stream);

/* The deterministic back-projection of lm_back(..., deterministic = 1, ...)
 * for callers that cannot allocate device memory or pass a workspace (a
 * plug-in whose host application owns all device memory, a real-time path
 * that must not allocate after start-up).  It allocates nothing: its scratch
 * is one fixed array inside the library, 2^22 voxels (64-bit sums) plus a
 * few words, 32 MiB + 256 B, held on every GPU that loads the library until
 * the process exits.  Grids above 2^22 voxels are rejected with
 * LM_ERR_NOMEM.  The result equals lm_back's deterministic result.  The first
 * call in a CUDA context looks up the array's device address in that
 * context (with its device current) and caches it under the context's id,
 * so a context that is destroyed and created again (cudaDeviceReset) gets a
 * fresh lookup; make the first call in each context before any stream
 * capture.  Every call
 * clears and reuses the same array, so calls that overlap on the GPU (other
 * streams, other threads, concurrent graph replays) race and must be
 * serialised by the caller.  The paper has no counterpart to this call. */
int lm_back_deterministic_noalloc(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                                  const lm_events* ev, const float* v, float* img, void* stream);

/* Sensitivity image sens = P^T 1 (Sec. "Listmode SPDHG": pre-computed once and
 * stored), i.e. the back-projection of ones over every canonical LOR and
 * every TOF bin, times lor_factor[l] (device float [lm_n_lor], NULL = 1).
 * The per-sample sum of the truncated bin weights over the bins is
 * evaluated in closed form (the bin integrals telescope).  Canonical LOR
 * order: transaxial pairs q in [0, n_xtal(n_xtal-1)/2): with
 * B = n_xtal*floor((n_xtal-1)/2), q < B -> c1 = q mod n_xtal,
 * c2 = (c1 + 1 + q div n_xtal) mod n_xtal; q >= B (even n_xtal) -> c1 = q-B,
 * c2 = c1 + n_xtal/2.  LOR l = (q*n_rings + r1)*n_rings + r2,
 * det1 = r1*n_xtal + c1, det2 = r2*n_xtal + c2.  sens is overwritten.
 * ws (device, may be NULL) of lm_sens_workspace_bytes() bytes speeds up
 * y-principal LORs. */
int64_t lm_n_lor(const lm_scanner* sc);
size_t lm_sens_workspace_bytes(const lm_grid* grid);
int lm_sens(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const float* lor_factor,
            float* sens, void* ws, size_t ws_bytes, void* stream);

/* ---- TV prior (Sec. "Numerical experiments": R(Kx) = ||Kx||_{2,1}) ------- */
/* K: unit-spacing forward differences with a Neumann boundary (last
 * difference 0), one component per axis with n_d > 1, in axis order;
 * components stored one after another ([ndim][V]).  lm_tv_ndim gives ndim. */
int lm_tv_ndim(const lm_grid* grid);
int lm_tv_grad(const lm_grid* grid, const float* x, float* g, void* stream);
/* d = div g = -K^T g. */
int lm_tv_div(const lm_grid* grid, const float* g, float* d, void* stream);
/* w <- beta prox_{R^*}(w / beta) = w / max(1, |w|/beta), per voxel over the
 * components (in place); beta = 0 sets w = 0. */
int lm_tv_prox(const lm_grid* grid, float* w, float beta, void* stream);
/* ---- image-space resolution model (Eq. (1): P includes the limited
 * spatial resolution) -------------------------------------------------- */
/* P = A G with A the projector above and G a separable Gaussian blur of full
 * width at half maximum fwhm (mm) on every axis with n_d > 1 (the paper gives
 * no kernel; this is the implemented one): sigma_d = fwhm/(2 sqrt(2 ln 2))/h_d
 * voxels, taps k = -r..r with r = floor(3 sigma_d + 1/2) (at most n_d - 1,
 * at most 31), weights exp(-k^2/(2 sigma_d^2)) normalised to sum 1, the
 * image mirrored about its outer faces.  G is symmetric with unit row sums,
 * so P^T = G A^T and P 1 = A 1; P^T 1 = G (lm_sens).  out = G x (out may
 * equal x); fwhm = 0 copies.  ws: device workspace of
 * lm_res_workspace_bytes(grid) bytes.  LM_ERR_INVALID_ARG for a kernel
 * wider than 31 taps per side. */
size_t lm_res_workspace_bytes(const lm_grid* grid);
int lm_res_apply(const lm_grid* grid, float fwhm, const float* x, float* out, void* ws, size_t ws_bytes,
                 void* stream);

/* ---- directional TV (the paper's second prior, Sec. "Numerical experiments") */
/* Only the part of the forward-difference vector perpendicular to the
 * gradient of a structural image v counts (after Ehrhardt & Betcke 2016):
 *   (K x)_j = P_j (grad x)_j,  P_j = I - xi_j xi_j^T,
 *   xi_j = (grad v)_j / sqrt(|(grad v)_j|^2 + eta^2)   (0 where both vanish),
 * so eta = 0 makes P_j the orthogonal projection perpendicular to (grad v)_j.
 * xi: device float [ndim][V] in the layout of lm_tv_grad (|xi_j| <= 1).
 * K^T q = grad^T (P q); ||K|| <= ||K_TV||.  lm_params.xi selects this prior
 * for LM-SPDHG.  lm_dtv_field: xi of v (eta >= 0); lm_dtv_grad: g = K x;
 * lm_dtv_div: d = -K^T g. */
int lm_dtv_field(const lm_grid* grid, const float* v, float eta, float* xi, void* stream);
int lm_dtv_grad(const lm_grid* grid, const float* xi, const float* x, float* g, void* stream);
int lm_dtv_div(const lm_grid* grid, const float* xi, const float* g, float* d, void* stream);
/* ||K|| by FP64 power iteration on K^T K from the checkerboard
 * (-1)^(ix+iy+iz), `iters` iterations; *out_host = sqrt of the last Rayleigh
 * quotient (never above ||K||).  Synchronous.  ws: device workspace of
 * lm_knorm_workspace_bytes() bytes. */
size_t lm_knorm_workspace_bytes(const lm_grid* grid);
int lm_knorm_fp64(const lm_grid* grid, int32_t iters, void* ws, size_t ws_bytes, double* out_host,
                  void* stream);

/* ---- event set-up (Alg. 2: event counts, sub lists) --------------------- */
/* Validates the events (0 <= det < n_det, det1 != det2, |tof| <= (n_bins-1)/2,
 * corr > 0, contam > 0), counts mu_e = number of events of the whole list in
 * the event's data bin (its unordered detector pair and TOF bin; footnote of
 * Sec. "Listmode SPDHG"), and writes the events in subset-contiguous order:
 * event e goes to subset e mod n_subsets, at rank e div n_subsets inside it
 * (Sec. "Listmode SPDHG": every n-th event to the n-th sub list).  Outputs
 * are device arrays of length ev->n: *_out (permuted fields) and mu_out
 * (uint16).  sub_off_host (host int64[n_subsets+1]) receives the subset
 * offsets.  Synchronous.  Returns LM_ERR_OUT_OF_RANGE / LM_ERR_DOMAIN on
 * invalid events (outputs undefined), LM_ERR_OUT_OF_RANGE if some mu > 65535.
 * ws: device workspace of lm_setup_workspace_bytes(n) bytes. */
size_t lm_setup_workspace_bytes(int64_t n_events);
int lm_event_setup(const lm_scanner* sc, const lm_tof* tof, const lm_events* ev, int32_t n_subsets,
                   int32_t* det1_out, int32_t* det2_out, int16_t* tof_out, float* corr_out,
                   float* contam_out, uint16_t* mu_out, int64_t* sub_off_host, void* ws,
                   size_t ws_bytes, void* stream);

/* ---- sinogram SPDHG (Alg. 1) ---------------------------------------------- */
/* The comparison method of the paper: SPDHG over every bin of the TOF
 * sinogram, empty bins included (Sec. "Memory-efficient SPDHG": y = 1 on
 * empty bins, Eq. (yinit) elsewhere).  lm_sino_setup lays the sinogram out as
 * an event list for lmspdhg_create with lm_params.sinogram = 1: bin b =
 * l * nb + (m + (nb-1)/2) of canonical LOR l (lm_sens's order) and signed TOF
 * bin m (nb = max(n_bins, 1)) becomes an event with det1/det2 of l's
 * canonical orientation, tof m, corr = lor_factor[l] (NULL = 1), contam =
 * s[b] (> 0, else LM_ERR_DOMAIN), and d_out = d[b] (the bin's count).  Bins
 * are grouped by view-based subsets: transaxial pair (c1, c2) has view
 * (c1 + c2) mod n_xtal (parallel LORs share it) and view v goes to subset
 * v mod n_subsets; inside a subset bins keep canonical order.
 * sub_off_host (host int64[n_subsets+1]) receives the offsets.  d, s:
 * device arrays of lm_sino_n_bins entries; outputs: device arrays of the
 * same length.  ws: device workspace of lm_sino_workspace_bytes bytes.
 * Synchronous. */
int64_t lm_sino_n_bins(const lm_scanner* sc, const lm_tof* tof);
size_t lm_sino_workspace_bytes(const lm_scanner* sc, int32_t n_subsets);
int lm_sino_setup(const lm_scanner* sc, const lm_tof* tof, int32_t n_subsets, const uint16_t* d, const float* s,
                  const float* lor_factor, int32_t* det1_out, int32_t* det2_out, int16_t* tof_out, float* corr_out,
                  float* contam_out, uint16_t* d_out, int64_t* sub_off_host, void* ws, size_t ws_bytes, void* stream);
/* Generated-geometry layout (lm_params.sinogram = 2), for sinograms too large
 * to hold as a bin list (the 3D scanner's 2.9e8 LORs x 41 bins): only the
 * counts are stored, in the order of lm_sino_setup; the event kernels compute
 * each bin's detectors and TOF bin from its index, with the LOR factor from
 * lm_params.sino_lorf and a flat contamination lm_params.sino_s.
 * lm_sino_count histograms the events of ev (validated like lm_event_setup;
 * LM_ERR_OUT_OF_RANGE for an invalid event or a bin above 65535 counts) into
 * d_out (device uint16, lm_sino_n_bins entries rounded up to an even number,
 * 4-byte aligned; overwritten), and writes the subsets' transaxial pairs
 * (q_out: device int32 [n_xtal (n_xtal - 1) / 2]) with their offsets (qoff_out:
 * device int64 [n_subsets + 1]) and the bin offsets (sub_off_host).  Same
 * workspace as lm_sino_setup.  Synchronous. */
int lm_sino_count(const lm_scanner* sc, const lm_tof* tof, int32_t n_subsets, const lm_events* ev, uint16_t* d_out,
                  int32_t* q_out, int64_t* qoff_out, int64_t* sub_off_host, void* ws, size_t ws_bytes, void* stream);

/* ---- LM-SPDHG state (Alg. 2) --------------------------------------------- */
typedef struct lm_state_s lm_state;

typedef struct {
    float beta;           /* prior weight, >= 0                                   */
    float gamma;          /* step-size ratio; <= 0: 3 / max(x0) (paper's choice)  */
    float rho;            /* 0 < rho < 1 (paper: 0.999)                           */
    double knorm;         /* ||K||; <= 0: FP64 power iteration (knorm_iters)      */
    int32_t knorm_iters;  /* iterations when knorm <= 0 (0: 1000)                 */
    int32_t n_subsets;    /* n >= 1                                               */
    int32_t deterministic;/* 1: fixed-point back-projection (bit-reproducible)    */
    int32_t kahan;        /* 1: compensated float32 accumulation of z             */
    int32_t group;        /* lanes per event in the event kernels: 8, 16 or 32;  */
                          /* 0: chosen at create by timing the forward projection */
                          /* of subset 0 with each width (autotuner)             */
    int32_t image_kernel; /* image passes: 0 auto (TMA-staged where the grid has */
                          /* nx, ny multiples of 4, nx >= 40, ny >= 36, with the  */
                          /* TV's dual step fused in, the directional TV's D =    */
                          /* P(w+ - w) staged from its dual step; plain loads     */
                          /* otherwise), 1 plain loads, 2 TMA-staged, 3 TMA-      */
                          /* staged data passes with plain prior passes (2 and 3: */
                          /* LM_ERR_INVALID_ARG if the grid does not allow it;    */
                          /* other values: LM_ERR_INVALID_ARG).  Same results.    */
    void* tile_buf;       /* device buffer of lmspdhg_tile_bytes() bytes for the  */
    size_t tile_bytes;    /* tile-binned projector of the data updates, or NULL:  */
                          /* used for TOF data in float-atomic mode (the batch    */
                          /* and the deterministic mode use the direct kernel).   */
                          /* The events' traversals are cut into segments per     */
                          /* 32x32x8 image tile at create/reinit; each data update*/
                          /* then projects tile by tile in shared memory.  Same   */
                          /* per-sample arithmetic, sums in another order.  If the*/
                          /* events need more segments than the buffer holds     */
                          /* (6 per event), the direct kernel is used.            */
    const float* xi;      /* directional TV prior (lm_dtv_field): device field    */
                          /* [ndim][V], referenced, must outlive the state; NULL  */
                          /* = TV.  The prior's dual step (with the field) runs  */
                          /* in the event kernel and stores D = P(w+ - w); the   */
                          /* image pass (TMA-staged where the grid allows) forms */
                          /* K^T(w+ - w) from D.  knorm may be the TV norm:      */
                          /* ||K_DTV|| <= ||K_TV||.                               */
    float res_fwhm;       /* image-space resolution model P = A G (lm_res_apply): */
                          /* FWHM in mm, 0 = none.  sens must then be G (lm_sens).*/
                          /* Float-atomic mode only (deterministic is rejected);  */
                          /* direct projector; not for batches.  Negative, NaN or */
                          /* more than 31 taps per side: LM_ERR_INVALID_ARG.      */
    int32_t sinogram;     /* 1: Alg. 1 (sinogram SPDHG): the events are the bins */
                          /* of lm_sino_setup and mu their counts d_b (0 allowed);*/
                          /* the dual step uses prox with S_b d_b and back-       */
                          /* projects y+ - y; the objective is Eq. (1) with the   */
                          /* sum of s.  0: Alg. 2 (listmode).  2: the same with  */
                          /* the bins' geometry generated (lm_sino_count): the   */
                          /* events' arrays may be NULL, mu = the counts.         */
    const int32_t* sino_q;   /* sinogram = 2: q_out of lm_sino_count               */
    const int64_t* sino_qoff;/* sinogram = 2: qoff_out of lm_sino_count            */
    const float* sino_lorf;  /* sinogram = 2: LOR factor [lm_n_lor] (NULL = 1)     */
    float sino_s;            /* sinogram = 2: flat contamination s_b > 0           */
    void* trav_buf;       /* device buffer of lmspdhg_trav_bytes() bytes for the  */
    size_t trav_bytes;    /* traversal-table data update, or NULL.  Used for TOF  */
                          /* data on 3D grids (n_y, n_z > 1, every axis < 2^15)  */
                          /* in float-atomic mode without the resolution model,  */
                          /* the tile-binned projector or sinogram bins; else    */
                          /* ignored.  At create/reinit every event's traversal  */
                          /* (the reading of Joseph's method: principal axis,    */
                          /* plane range, secondary and TOF coordinates, sample  */
                          /* length), 1/(P^LM 1)_e and 1/mu_e are stored (40 B   */
                          /* per event); each data update then reads them        */
                          /* instead of setting the traversals up again.  Same   */
                          /* per-sample arithmetic as the direct kernel; S_e and */
                          /* (y+ - y)/mu from the stored reciprocals.  Batches   */
                          /* (lmspdhg_batch_*) run their frames' tables too.     */
                          /* With group = 0 the autotuner also times the direct  */
                          /* event kernel on one subset and keeps the faster     */
                          /* projector unless trav_keep is set.                  */
    int32_t shard;        /* 1: event sharding of one frame over several states  */
                          /* (one per GPU), each holding a slice of every        */
                          /* subset's events (mu counted over the whole list:   */
                          /* lm_event_setup on the whole list, then a slice of   */
                          /* each subset).  The data term is a sum over events,  */
                          /* so each update's dz is the sum of the states'       */
                          /* partial back-projections: updates then run through  */
                          /* lmspdhg_shard_begin / _finish with the caller's sum */
                          /* of lmspdhg_shard_buffer over the states in between; */
                          /* prior updates and primal steps are replicated.      */
                          /* Float-atomic mode; not with the resolution model,   */
                          /* the tile-binned projector or sinogram bins          */
                          /* (LM_ERR_INVALID_ARG).  0: the frame's events all    */
                          /* belong to this state.                               */
    int32_t epoch_kernel; /* how lmspdhg_epoch runs its 2n updates: 0 auto, 1 a  */
                          /* captured graph of per-update launches, 2 one        */
                          /* persistent cooperative launch per epoch (2D grids,  */
                          /* float-atomic mode, TV prior, direct projector, no   */
                          /* resolution model or sinogram bins; else             */
                          /* LM_ERR_INVALID_ARG).  Auto takes 1: on the 2D frame */
                          /* the graph is faster (0.65 against 0.86 ms/epoch).    */
                          /* Its grid-wide barriers wait at most one second; a   */
                          /* wait that gives up ends the kernel and the next     */
                          /* lmspdhg_objective_fp64 returns LM_ERR_TIMEOUT.      */
    int32_t trav_keep;    /* 1: keep the traversal table whenever trav_buf serves */
                          /* the frame (no timing against the direct kernel;     */
                          /* lmspdhg_tuning_projectors then reports 0 for it).   */
                          /* 0: the faster of the two, as measured at create.    */
} lm_params;

/* Bytes of the optional traversal-table buffer (lm_params.trav_buf): 40 per
 * event (plus alignment); 0 for a grid the table does not serve. */
size_t lmspdhg_trav_bytes(const lm_grid* grid, int64_t n_events);

/* Bytes of the optional tile-binned projector buffer (lm_params.tile_buf):
 * about 136 per event plus per-tile tables. */
size_t lmspdhg_tile_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets);

/* Device bytes the state needs (images, duals, per-event y and scratch) with
 * the TV prior.  lmspdhg_state_bytes_ex: for the given parameters (the
 * directional TV prior, lm_params.xi, adds ndim images); lmspdhg_create
 * checks the buffer against it. */
size_t lmspdhg_state_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets,
                           int32_t deterministic);
size_t lmspdhg_state_bytes_ex(const lm_grid* grid, int64_t n_events, int32_t n_subsets, const lm_params* params);

/* Initialise Alg. 2 (duals, z, step sizes) on events already in subset-contiguous
 * order (from lm_event_setup; the arrays are referenced, not copied, and
 * must outlive the state):
 *   y_e = 1 - mu_e / ((P^LM x0)_e + s_e)                      (Eq. yinit)
 *   z = zbar = P^T 1 + (P^LM)^T((y - 1)/mu) + K^T w, w = 0
 *     (= P^T applied to the sinogram that is 1 on empty bins and Eq. yinit
 *      elsewhere; the printed minus sign of the z initialisation is read as this plus)
 *   T = min_k T_k with T_k = gamma^-1 rho p_k / (P^T 1 / n) for data subsets
 *   and T_{n+1} = gamma^-1 p_{n+1} rho / ||K||;  S_e = gamma rho / (P^LM 1)_e
 *   (Eq. lm_stepsizes), S_{n+1} = gamma rho / ||K||; p_k = 1/(2n), p_{n+1} = 1/2.
 * sens: device P^T 1 (lm_sens), referenced.  x0: device image >= 0 (copied).
 * sub_off_host: host int64[n+1].  state_buf: device buffer of
 * lmspdhg_state_bytes() bytes owned by the caller.  Synchronous (reads
 * max(x0), min(x0) and, if asked for, ||K||).  *out receives a host handle;
 * free it with lmspdhg_destroy.  Invalid parameters (NULL pointers, subset
 * offsets, beta, rho, image_kernel, res_fwhm, sinogram options, a buffer
 * smaller than lmspdhg_state_bytes_ex) are rejected on the host before any
 * device call. */
int lmspdhg_create(lm_state** out, const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                   const lm_events* ev_perm, const uint16_t* mu, const int64_t* sub_off_host,
                   const float* sens, const float* x0, const lm_params* params, void* state_buf,
                   size_t state_bytes, void* stream);

/* Run `count` updates of the Alg. 2 loop (x <- proj(x - T zbar); selected
 * update; z <- z + dz; zbar <- z + dz/p_i).  seq_host: host uint16[count],
 * value i < n selects data subset i, value n selects the prior.  Any count. */
int lmspdhg_updates(lm_state* st, const uint16_t* seq_host, int32_t count, void* stream);

/* One epoch = 2n updates, replayed from a CUDA graph captured on first use
 * (the selection is read on the device, so one graph serves every sequence).
 * seq_host: host uint16[2n]. */
int lmspdhg_epoch(lm_state* st, const uint16_t* seq_host, void* stream);

/* Copies (device to device) the x used by the most recent update (x0 before
 * any update), the dual list y (subset-contiguous order), z (with its
 * compensation added) and w ([ndim][V]). */
int lmspdhg_get_x(lm_state* st, float* x_out, void* stream);
int lmspdhg_get_y(lm_state* st, float* y_out, void* stream);
int lmspdhg_get_z(lm_state* st, float* z_out, void* stream);
int lmspdhg_get_w(lm_state* st, float* w_out, void* stream);

/* Objective of Eq. (1) in listmode form at the x of lmspdhg_get_x, without
 * the constant sum of s over all bins:
 *   <P^T 1, x> - sum_e log((P^LM x)_e + s_e) + beta ||Kx||_{2,1},
 * projections in float32, logs and sums in FP64 (fixed reduction order).
 * Synchronous. */
int lmspdhg_objective_fp64(lm_state* st, double* out_host, void* stream);

/* Number of updates run so far and the state's parameters (gamma, knorm
 * as resolved at create). */
int lmspdhg_info(lm_state* st, int64_t* n_updates, double* gamma, double* knorm);

/* The event-kernel width in use and, if it was autotuned, the measured
 * forward-projection times of subset 0 (ms) for widths 8, 16, 32 (else 0). */
int lmspdhg_tuning(lm_state* st, int32_t* group, double* ms3);

/* Re-initialise the state (as lmspdhg_create initialises Alg. 2) for the
 * current contents of the referenced event arrays and a new x0, keeping the
 * buffers and the captured epoch graph: the events may have been overwritten
 * with another frame of the same size and subset split.  Synchronous. */
int lmspdhg_reinit(lm_state* st, const float* x0, void* stream);

/* Runs `count` (1..2n) updates like lmspdhg_updates, recording CUDA events on
 * `stream` around every kernel; ms4/n4 (host, 4 entries) receive the summed
 * milliseconds and launch counts of: [0] data-update event kernels, [1] prior
 * dual-step kernels, [2] image passes after data updates, [3] image passes
 * after prior updates.  Synchronous. */
int lmspdhg_profile(lm_state* st, const uint16_t* seq_host, int32_t count, double* ms4, int64_t* n4,
                    void* stream);

/* ---- event sharding of one frame (lm_params.shard = 1) -------------------
 * Alg. 2's data update of subset i adds dz = (P^LM_{N_i})^T ((y+ - y)/mu)
 * over the subset's events, a sum that splits over any partition of the
 * events; the dual step of each event needs only its own projection.  A
 * frame's events can therefore be spread over states (ranks) that each hold
 * a slice of every subset and a full copy of the image variables: after
 * each rank's event kernels the ranks sum their partial dz (all-reduce),
 * and every rank applies the same image pass.  The initialisation's
 * back-projection z0 = P^T 1 + (P^LM)^T((y - 1)/mu) splits the same way.
 * Protocol per state:
 *   lmspdhg_create (shard = 1): y of the state's events; its partial
 *     back-projection of the initialisation is left in the exchange buffer;
 *   the caller sums the buffers of all states into each (an all-reduce);
 *   lmspdhg_shard_init_finish: z, T and the first primal step;
 *   per update: lmspdhg_shard_begin(sel) (for a data selection the state's
 *     partial dz lands in the buffer), the caller's sum over states (data
 *     selections only), lmspdhg_shard_finish.
 * lmspdhg_epoch / lmspdhg_updates / lmspdhg_profile are rejected on a shard
 * state (LM_ERR_INVALID_ARG), as are calls out of this order.  The buffer is
 * V floats of device memory inside the state buffer (valid while the state
 * lives); its content between begin and finish is the state's partial dz. */
int lmspdhg_shard_buffer(lm_state* st, float** dz_out);
int lmspdhg_shard_init_finish(lm_state* st, void* stream);
int lmspdhg_shard_begin(lm_state* st, uint16_t sel, void* stream);
int lmspdhg_shard_finish(lm_state* st, void* stream);

/* The FP64 objective's parts: out4[0] = <P^T 1, x>, out4[1] = ||K x||_{2,1},
 * out4[2] = sum_e w_e log((P^LM x)_e + s_e) over this state's events,
 * out4[3] = sum of s over sinogram bins (0 for listmode).  The objective is
 * out4[0] - out4[2] + beta out4[1] + out4[3]; with event sharding out4[2]
 * is summed over the states.  Synchronous. */
int lmspdhg_objective_parts_fp64(lm_state* st, double* out4, void* stream);

/* The autotuner's comparison of the projectors (lm_params.trav_buf with
 * group = 0): the data update of subset 0 with the best traversal-table
 * variant and with the best direct-kernel width, in ms (0 when not
 * measured); the state keeps the faster one (lmspdhg_projector), or the
 * table when lm_params.trav_keep is set (the direct kernel is then not
 * timed and direct_ms is 0). */
int lmspdhg_tuning_projectors(lm_state* st, double* table_ms, double* direct_ms);

/* Failure injection for the persistent epoch kernel (lm_params.epoch_kernel
 * = 2): with flag != NULL (device memory), its first block waits for *flag
 * != 0 before the first update, at most one second; if nothing sets the
 * flag, that wait and the other blocks' barrier waits give up, the kernel
 * returns and lmspdhg_objective_fp64 reports LM_ERR_TIMEOUT (lmspdhg_reinit
 * clears the condition).  NULL removes the gate. */
int lmspdhg_set_gate(lm_state* st, const unsigned* flag);

/* How the state's epochs run: 1 a graph of per-update launches, 2 one
 * persistent launch per epoch. */
int lmspdhg_epoch_kernel(lm_state* st, int32_t* kind);

/* Which image-pass kernel the state uses (lm_params.image_kernel): 1 plain
 * loads, 2 TMA-staged (the TV's dual step fused in; the directional TV's
 * dual step stays in the event kernel and the pass stages its D), 3
 * TMA-staged data passes with plain prior passes. */
int lmspdhg_image_kernel(lm_state* st, int32_t* kind);

/* Which projector the data updates use: 1 direct event kernel, 2 tile-binned
 * (lm_params.tile_buf), 3 traversal table (lm_params.trav_buf); *n_segments
 * receives the number of tile segments of the current events (0 for the
 * others). */
int lmspdhg_projector(lm_state* st, int32_t* kind, int64_t* n_segments);

/* Frees the host handle, its captured epoch graph and its capture stream.
 * The state buffer, the events and the images it referenced stay the
 * caller's (no device memory is freed); work already queued on the caller's
 * stream must be complete or ordered before the buffer is reused.  NULL is
 * a no-op.  Returns LM_OK. */
int lmspdhg_destroy(lm_state* st);

/* ---- listmode EM-TV: the warm start x0 (Alg. 3) ------------------------- */
/* The listmode experiments start LM-SPDHG from one pass of listmode EM-TV
 * over the n subsets (Alg. 3, Sec. "Numerical experiments").  For subsets
 * i = 0, 1, ..., n-1 in turn, with g = P^T 1 (sens):
 *   z = x n / g * (P^LM_{N_i})^T (1 / (P^LM_{N_i} x + s_{N_i}))   (EM step)
 *   w = g / (beta x)
 *   x = argmin_{u >= 0} sum_j w_j/2 (u_j - z_j)^2 + ||K u||_{2,1}  (weighted TV denoising)
 * Readings (the paper leaves them open): the EM step's forward projection
 * uses the current x; z_j = 0 where g_j = 0; voxels with x_j = 0 or g_j = 0
 * are held at 0 (w_j = 0); the denoising problem is solved by `pdhg_iters`
 * iterations of the accelerated primal-dual algorithm of Chambolle & Pock
 * (2011, their Alg. 2) from u = z, q = 0, tau_0 = sigma_0 = 0.99/knorm,
 * with the uniform convexity gam = min w_j over the free voxels:
 *   q <- q / max(1, |q|) after q += sigma K ubar;  u+ = max(0, (u - tau K^T q
 *   + tau w z) / (1 + tau w));  theta = 1/sqrt(1 + 2 gam tau);  tau *= theta;
 *   sigma /= theta;  ubar = u+ + theta (u+ - u).
 * beta = 0 makes x = z (listmode OSEM).  float32 images and float atomics
 * (the back-projection's order of additions varies between runs).
 *
 * lm_emtv_epoch: ev_perm holds the events in subset-contiguous order
 * (lm_event_setup's det/tof/corr/contam output; mu unused) with host int64
 * offsets sub_off_host[n_subsets+1] (0 .. n, non-decreasing).  sens, x:
 * device float images; x (in/out) >= 0.  beta >= 0; pdhg_iters in
 * [0, 10000]; knorm = ||K|| (lm_knorm_fp64) or an upper bound, > 0.
 * ws: device workspace of lm_emtv_workspace_bytes(grid) bytes, 256-byte
 * aligned.  Asynchronous on `stream`; LM_ERR_NOMEM for a short workspace,
 * LM_ERR_INVALID_ARG for the other argument errors (nothing is queued). */
size_t lm_emtv_workspace_bytes(const lm_grid* grid);
int lm_emtv_epoch(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev_perm,
                  const int64_t* sub_off_host, int32_t n_subsets, const float* sens, float* x, float beta,
                  int32_t pdhg_iters, double knorm, void* ws, size_t ws_bytes, void* stream);
/* The EM step alone over the events of ev (one subset):
 * z = x n_subsets / sens * (P^LM)^T (1 / (P^LM x + s)), z overwritten
 * (device float image, 0 where sens = 0).  Same workspace. */
int lm_emtv_em_step(const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof, const lm_events* ev,
                    int32_t n_subsets, const float* sens, const float* x, float* z, void* ws, size_t ws_bytes,
                    void* stream);
/* The weighted TV denoising alone: u (device float image, overwritten) after
 * `iters` iterations from u = z; voxels with w_j <= 0 are held at 0.  Same
 * workspace. */
int lm_emtv_denoise(const lm_grid* grid, const float* z, const float* w, float* u, int32_t iters, double knorm,
                    void* ws, size_t ws_bytes, void* stream);

/* ---- batched epochs of several frames ----------------------------------- */
/* A batch advances every occupied slot (an lm_state) by one epoch of Alg. 2
 * in one captured CUDA graph: each update is one event kernel whose work
 * items span the events of every frame's selected subset (or the voxels of
 * its prior step) and one image pass over all frames' tiles, so small
 * frames share the GPU instead of each leaving most of it idle.  The states
 * of a batch must share the grid, TOF kernel, subset count, crystal count
 * and mode (deterministic / compensated); each keeps its own events, duals,
 * images and selection sequence.  Results equal lmspdhg_epoch on each state
 * alone (bit for bit in deterministic mode; within float32 rounding of the
 * atomic back-projection otherwise).  Slots are filled or emptied between
 * epochs (continuous batching); the graph does not change.
 * buf: device workspace of lmspdhg_batch_bytes(capacity, n_subsets) bytes;
 * capacity <= 64. */
typedef struct lm_batch_s lm_batch;
size_t lmspdhg_batch_bytes(int32_t capacity, int32_t n_subsets);
int lmspdhg_batch_create(lm_batch** out, int32_t capacity, int32_t n_subsets, void* buf, size_t bytes,
                         void* stream);
/* Puts `st` into `slot` (NULL empties it).  A state joins after an even
 * number of updates (e.g. after create/reinit or whole epochs) and may not
 * occupy two slots.  Synchronous. */
int lmspdhg_batch_set(lm_batch* b, int32_t slot, lm_state* st, void* stream);
/* One epoch for every occupied slot; seqs_host: host uint16[capacity][2n]
 * (rows of empty slots are ignored). */
int lmspdhg_batch_epoch(lm_batch* b, const uint16_t* seqs_host, void* stream);
int lmspdhg_batch_destroy(lm_batch* b);

/* ---- reconstruction server: continuous batching of frames ---------------- */
/* The paper reconstructs one frame at a time; a server of many short frames
 * (dynamic or gated studies, Sec. "Discussion") has no counterpart there.
 * A server owns one lm_batch and a worker thread.  Frames are queued by
 * lm_server_submit (host arrays, copied) and admitted in arrival order when
 * a slot is free and the caller's device pool has room for the frame
 * (lm_server_frame_bytes; first-fit with coalescing); admission uploads the
 * events, runs lm_event_setup and lmspdhg_create from the uniform image
 * x0_value.  Every loop of the worker advances all admitted frames by one
 * epoch of their own selection sequence in one batched launch, then retires
 * the frames that finished (x and the FP64 objective copied to the host,
 * pool memory released), so frames join and leave between epochs while the
 * others keep running.  A frame's result equals a lone lmspdhg run of it
 * (bit for bit in deterministic mode).  */
typedef struct lm_server_s lm_server;

typedef struct {
    float beta;             /* TV weight                                        */
    float rho;              /* step-size safety factor (paper: 0.999)           */
    double knorm;           /* ||K|| (> 0; from lm_knorm_fp64)                  */
    int32_t n_subsets;      /* data subsets n                                   */
    int32_t epochs;         /* epochs per frame (>= 1)                          */
    int32_t max_slots;      /* frames on the GPU at once (1..64)                */
    int32_t deterministic;  /* fixed-point back-projection                      */
    int32_t kahan;          /* compensated z                                    */
    int32_t group;          /* lanes per event (8, 16, 32; 0: 32)               */
    int64_t max_events;     /* largest frame accepted                           */
} lm_server_config;

/* Pool bytes one admitted frame of n_events holds. */
size_t lm_server_frame_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets, int32_t deterministic);

/* sens: device P^T 1, referenced.  pool: device memory owned by the caller
 * (must outlive the server); it must hold the event set-up workspace of
 * max_events, the batch workspace and one frame of max_events, else
 * LM_ERR_NOMEM.  The server runs on the calling thread's current device. */
int lm_server_create(lm_server** out, const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                     const float* sens, const lm_server_config* cfg, void* pool, size_t pool_bytes);

/* Queues one frame.  Host arrays of n events (tof may be NULL for non-TOF,
 * corr NULL for all ones); x0_value > 0; seqs_host: host
 * uint16[epochs][2 n_subsets], the frame's selection sequence (values <=
 * n_subsets).  n > max_events gives LM_ERR_NOMEM.  Returns at once; invalid
 * events are reported by lm_server_wait. */
int lm_server_submit(lm_server* s, const int32_t* det1, const int32_t* det2, const int16_t* tof,
                     const float* corr, const float* contam, int64_t n, float x0_value,
                     const uint16_t* seqs_host, int64_t* ticket);

/* Waits at most timeout_ms for a ticket: LM_ERR_TIMEOUT if unfinished (the
 * ticket stays valid), else the frame's status; on LM_OK fills x_host
 * (float[V], may be NULL), *objective and *latency_ms (submit to retire) and
 * the ticket is released. */
int lm_server_wait(lm_server* s, int64_t ticket, float* x_host, double* objective, double* latency_ms,
                   int32_t timeout_ms);

/* Frames finished, on the GPU now, queued; pool bytes in use; the most
 * frames that were on the GPU together so far.  NULL outputs are skipped. */
int lm_server_stats(lm_server* s, int64_t* completed, int64_t* in_flight, int64_t* queued, size_t* pool_used,
                    int64_t* max_in_flight);

/* Stops the worker after its current epoch and frees everything; queued and
 * unfinished frames are dropped. */
int lm_server_destroy(lm_server* s);

/* ---- measurement utilities (no counterpart in the paper) ---------------- */
/* Kernels launched by this library in this process so far (a replayed
 * epoch graph counts each of its kernel nodes). */
int64_t lm_kernel_launches(void);

/* The benchmark's own measurement utilities (throughput probes, traversal
 * statistics) are declared in lm_measure.h. */

#ifdef __cplusplus
}
#endif
#endif /* LMSPDHG_H */
