// Internal host-side declarations shared by the library's translation units.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "../../include/lmspdhg.h"
#include "lm_device.cuh"

namespace lmh {

void set_error(const char* fmt, ...);
void clear_error();

#define LM_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ::lmh::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return LM_ERR_CUDA;                                                                \
        }                                                                                      \
    } while (0)

#define LM_CHECK(cond, code, ...)             \
    do {                                      \
        if (!(cond)) {                        \
            ::lmh::set_error(__VA_ARGS__);    \
            return (code);                    \
        }                                     \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Validates the descriptors and fills the device geometry.
int make_geo(const lm_scanner* sc, const lm_grid* g, const lm_tof* tof, lmk::Geo& G, bool need_scanner);
int check_grid(const lm_grid* g);
int tv_ndim(const lm_grid* g);
inline int64_t nvox(const lm_grid* g) { return (int64_t)g->n[0] * g->n[1] * g->n[2]; }
inline size_t align_up(size_t v, size_t a = 256) { return (v + a - 1) / a * a; }

int num_sms();

// Intervals of the tabulated TOF kernel (bin-integrated Gaussian on [-W, W]).
constexpr int TOF_TAB_N = 4096;
// Fills tab[0..TOF_TAB_N] (host) with w(tau) at tau = -W + k 2W/TOF_TAB_N.
void tof_table(const lm_tof* tof, float* tab);

// TOF weight of the event's bin from the (shared-memory) table of the
// bin-integrated Gaussian w(tau), tau in [-W, W] on TOF_TAB_N intervals,
// linear interpolation; the 3-sigma cut is the same test as tof_weight's.
// inv_dt = TOF_TAB_N / (2W).
__device__ __forceinline__ float tof_weight_tab(const lmk::Geo& G, const float* tab, float inv_dt, float tau)
{
    if (fabsf(tau) > G.W) return 0.0f;
    const float u = fminf(fmaxf((tau + G.W) * inv_dt, 0.0f), (float)TOF_TAB_N);
    const int k = min((int)u, TOF_TAB_N - 1);
    const float f = u - (float)k;
    const float a = tab[k];
    return fmaf(f, tab[k + 1] - a, a);
}

// One sample of a traversal with the TOF weight from the table: base voxel
// index and the four bilinear weights times TOF weight times sample length.
template <bool TWO_D>
__device__ __forceinline__ bool sample_tab(const lmk::Geo& G, const lmk::Lor& L, const float* tab, float inv_dt, int i, lmk::Smp& s)
{
    const float fi = (float)i;
    const float tau = fmaf(fi, L.dtau, L.tau0);
    const float wt = L.step * tof_weight_tab(G, tab, inv_dt, tau);
    if (wt == 0.0f) return false;
    const float ua = fmaf(fi, L.sa, L.ua0);
    const float fla = floorf(ua);
    const int ia = (int)fla;
    const float fa = ua - fla;
    const float wa0 = (ia >= 0 && ia < L.nA) ? (1.0f - fa) : 0.0f;
    const float wa1 = (ia + 1 >= 0 && ia + 1 < L.nA) ? fa : 0.0f;
    if (TWO_D) {
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
        const float wtA0 = wt * wa0, wtA1 = wt * wa1;
        s.w0 = wtA0 * wb0;
        s.w1 = wtA1 * wb0;
        s.w2 = wtA0 * wb1;
        s.w3 = wtA1 * wb1;
        return (s.w0 != 0.0f) || (s.w1 != 0.0f) || (s.w2 != 0.0f) || (s.w3 != 0.0f);
    }
}

// Strides and extents of the traversal for principal axis k (set-up results
// travel between lanes as k plus the affine coefficients).
__device__ __forceinline__ void lor_strides(const lmk::Geo& G, int k, bool has_yf, lmk::Lor& L)
{
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    if (k == 0) {
        L.sk = 1; L.sA = nx; L.sB = nx * ny; L.nA = ny; L.nB = nz; L.yf = 0;
    } else if (k == 1) {
        L.nA = nx; L.nB = nz;
        if (has_yf) { L.sk = 1; L.sA = ny; L.sB = nx * ny; L.yf = 1; }
        else { L.sk = nx; L.sA = 1; L.sB = nx * ny; L.yf = 0; }
    } else {
        L.sk = nx * ny; L.sA = 1; L.sB = nx; L.nA = nx; L.nB = ny; L.yf = 0;
    }
}

// Kernel launches issued by the library (graph replays count their nodes).
void count_launch(int64_t n = 1);
int64_t launch_total();

// ---- event kernels (lm_project.cu) ----
enum EvMode {
    EV_FWD = 0,        // out[e] = corr*J(x)
    EV_BACK = 1,       // acc += corr*v[e]*J^T          (float atomics)
    EV_BACK_FX = 2,    // acci += round(vin[e]*J^T*2^E) (vin already includes corr)
    EV_DATA = 3,       // fused data update (float atomics)
    EV_DATA_FX1 = 4,   // data update forward part: y <- y+, out[e] = corr*v, max|.|
    EV_YINIT = 5,      // y = 1 - mu/(corr*J(x)+s); acc += corr*(y-1)/mu*J^T
    EV_YINIT_FX1 = 6,  // y init, out[e] = corr*(y-1)/mu, max|.|
    EV_ABSMAX = 7,     // max |corr*v[e]|
    EV_COUNT = 8,      // traversal statistics: samples and neighbour touches
    EV_EM = 9          // subset EM step (Alg. 3): acc += corr * J^T / (corr*J(x) + s)
};

struct EvArgs {
    lmk::Geo G;
    const float* x_std;
    const float* x_yf;
    float* acc_std;
    float* acc_yf;
    unsigned long long* acci_std;
    unsigned long long* acci_yf;
    const int32_t* det1;
    const int32_t* det2;
    const int16_t* tof;
    const float* corr;
    const float* contam;
    const uint16_t* mu;
    float* y;
    const float* vin;
    float* out;
    int64_t e_begin, e_end;
    // selection read on the device (epoch graphs): if seq != nullptr the
    // range is subset seq[u] and a prior selection (seq[u] == n_subsets)
    // runs the prior's dual step instead.
    const uint16_t* seq;
    int u;
    const int64_t* sub_off;
    int n_subsets;
    float gamma_rho;
    unsigned* maxbits;          // float bits of max |value| (non-negative floats order as uints)
    float stepmax;
    unsigned long long* queue;  // dynamic chunk counter (self-resetting)
    unsigned* done;
    int chunk;                  // events per warp grab (1..32)
    // prior dual step (selection == n_subsets)
    const float* px;            // x (std)
    const float* w_cur[2];      // indexed by wpar[u]
    float* w_nxt[2];
    const int* wpar;
    float s_prior;              // S_{n+1} = gamma rho / ||K||
    float beta;
    int ndim;
    const float* tof_tab;       // device table (TOF_TAB_N + 1 floats) or nullptr (erf per sample)
    int group;                  // lanes per event: 8, 16 or 32 (0 = 16)
    // batched epochs: both x buffers (index = update parity) and the scale slots
    const float* xb[2];
    const float* xbyf[2];
    unsigned* maxbits_base;
    int prior_fused;            // 1: the prior's dual step runs inside the TMA image pass instead
    int prior_only;             // 1: data selections are left to the tile-binned projector
    int acc_pairs;              // 1: acc_std / acc_yf hold (voxel j, voxel j + nx*ny) float pairs
    const float* xi;            // directional TV field [ndim][V], or nullptr (TV)
    float* dtv_d;               // directional TV: P (w+ - w) of the prior's dual step [ndim][V], or nullptr
    int sino;                   // 1: the events are sinogram bins, mu their counts d_b (Alg. 1);
                                // 2: the same, with each bin's geometry computed from its index
    const int32_t* g_q;         // sino 2: transaxial pairs of every subset, subset by subset
    const int64_t* g_qoff;      // sino 2: [n_subsets + 1] offsets into g_q
    const float* g_lorf;        // sino 2: per-LOR factor [n_lor] or nullptr (1)
    float g_s;                  // sino 2: flat contamination s_b
    int g_rings, g_xtal, g_nb;  // sino 2: scanner rings, crystals per ring, TOF bins (>= 1)
};

// Batched multi-frame epochs: per-frame argument tables in device memory.
constexpr int BATCH_MAX = 64;

struct BatchEvArgs {
    const EvArgs* slots;        // [cap]
    const int* active;          // [cap]
    const uint16_t* seqs;       // [cap][seq_stride]
    int seq_stride;
    int cap;
    int u;
    int slot0;                  // scale slot of update u: (slot0 + u) & 1
    unsigned long long* queue;  // self-resetting work counter
    unsigned* done;
    const float* tof_tab;       // shared TOF table (all frames have the same TOF kernel) or nullptr
    float tof_W;
    int vitem;                  // voxels per prior work item
};
// One epoch of a 2D frame in one cooperative launch (float accumulators,
// TV prior): per update the data update's event chunks or the prior's dual
// step, a grid-wide barrier, the image pass voxel by voxel, a barrier.
struct PersistArgs {
    EvArgs ev;                 // event and prior arguments (x set per update)
    const float* xs[2];        // x (std), by buffer
    float* xw[2];              // the same, written
    float* xyf[2];             // y-fastest copies
    const uint16_t* seq;       // device, count entries
    int count;
    int xpar0;                 // buffer holding the x of update 0
    float* z;
    float* zc;
    const float* T;
    int kahan;
    float inv_p_data, inv_p_prior;
    unsigned* bar;             // [2] arrival count, generation (zeroed before the launch)
    unsigned* err;             // bit 2: a barrier or the gate gave up waiting
    const unsigned* gate;      // nullptr, or a flag block 0 waits for (bounded) before update 0
};
bool persist_supported();
int persist_grid(int group);
int launch_persist_epoch(const PersistArgs& p, int group, int grid, cudaStream_t st);

int launch_events_batch(int mode, bool two_d, int group, const BatchEvArgs& b, int grid, cudaStream_t st);
int ev_batch_grid(int mode, bool two_d, int group);  // group 0: smallest over 8/16/32

int launch_events(int mode, bool two_d, const EvArgs& a, int grid, cudaStream_t st);
int ev_grid(int mode, bool two_d);  // smallest over the group widths
int ev_grid_g(int mode, bool two_d, int group);

// ---- tile-binned projector (lm_tile.cu) ----
constexpr int TL_TX = 32, TL_TY = 32, TL_TZ = 8;  // image tile (2D grids: TL_TZ -> 1)
constexpr int TL_CH = 512;                        // segments per work item
constexpr int TL_SEGCAP = 6;                      // segment capacity per event

struct TileItem {
    int tile;
    unsigned start;
    int count;
    int pad;
};

struct TileArgs {
    lmk::Geo G;
    int ntile[3];
    int tz;
    int64_t n_tiles;
    int n_subsets;
    const float* tof_tab;
    // events (subset-contiguous)
    const int32_t* det1;
    const int32_t* det2;
    const int16_t* tofb;
    const float* corr;
    const float* contam;
    const uint16_t* mu;
    float* y;
    const int64_t* sub_off;
    // per-frame binning
    float4* evp;         // 2 per event: (ua0, sa, ub0, sb), (tau0, dtau, step, k | 4 if valid)
    float* p1;           // (P^LM 1)_e
    unsigned* seg_off;   // [N+1] first segment of each event (event order)
    uint2* seg;          // tile-sorted segments: (event, first plane | planes << 16)
    unsigned* seg_pos;   // [segments] tile-sorted position of the event's s-th segment
    float* part;         // forward partial sum of each tile-sorted segment
    TileItem* items;     // work items, subset by subset
    int* item_off;       // [n+1]
    int max_items;       // most items of one subset
    // one update
    const uint16_t* seq;
    int u;
    const float* x;      // std layout
    float* acc;          // std-layout accumulator
    float* v;            // c_e (y+ - y)/mu per event
    float gamma_rho;
};

struct TileLayout {
    size_t evp, p1, seg_off, nseg, seg, seg_pos, part, tiles, items, item_off, bsums, bblocks, bhist, total;
    int64_t cap, max_items, max_bblocks;
};
constexpr int TL_EPB = 4096;        // events per binning block
constexpr int TL_MAX_TILES = 16384; // larger tile grids use the direct kernel
void tile_geometry(const lm_grid* g, int ntile[3], int* tz, int64_t* n_tiles);
TileLayout tile_layout(const lm_grid* g, int64_t N, int n_subsets);
// Bins the events (synchronous); LM_ERR_NOMEM if they need more segments than the layout holds.
int tile_build(TileArgs& A, const TileLayout& L, char* base, int64_t N, const std::vector<int64_t>& sub_off_h,
               bool two_d, cudaStream_t st, int64_t* n_segments);
void tile_attributes();
int launch_tile_update(const TileArgs& A, bool two_d, cudaStream_t st);

// ---- traversal-table data update (lm_table.cu) ----
// Per event (subset-contiguous order): the traversal of reading 1,
// 1/(P^LM 1)_e and 1/mu_e, computed once per state.
struct TravLayout {
    size_t r0, r1, meta, total;
};
TravLayout trav_layout(const lm_grid* g, int64_t N);
bool trav_capable(const lm_grid* g);  // 3D grids with n_y > 1, every axis < 2^15

struct TabArgs {
    lmk::Geo G;
    // table
    const float4* r0;      // (ua0, sa, ub0, sb)
    const float4* r1;      // (tau0, dtau, step, 1/(P^LM 1)_e)
    const int2* meta;      // (i0 | cnt << 15 | k << 30, bits of 1/mu_e); cnt = 0: inert event
    // events
    const float* corr;
    const float* contam;
    const uint16_t* mu;
    float* y;
    // images: the x the update gathers from, both layouts; z-paired accumulators (see EvArgs)
    const float* x_std;
    const float* x_yf;
    float* acc_std;
    float* acc_yf;
    const float* tof_tab;  // TOF_TAB_N + 1 floats
    // selection
    const uint16_t* seq;
    int u;
    const int64_t* sub_off;
    int n_subsets;
    int64_t e_begin, e_end;  // used when seq == nullptr
    float gamma_rho;
    unsigned long long* queue;
    unsigned* done;
    int phase;             // 0: x-principal events only, 1: the others, -1: all
    // batched epochs: the image of update u is in buffer u & 1
    const float* xs[2];
    const float* xyfs[2];
};

// The data updates of every active frame of a batch (frames with tables).
struct BatchTabArgs {
    const TabArgs* slots;       // [cap]
    const int* active;          // [cap]
    const uint16_t* seqs;       // [cap][seq_stride]
    int seq_stride;
    int cap;
    int u;
    unsigned long long* queue;  // self-resetting work counter
    unsigned* done;
    const float* tof_tab;       // the batch's TOF table
    float tof_W;
};
int launch_table_batch(const BatchTabArgs& b, int variant, int grid, cudaStream_t st);
int trav_build(const lmk::Geo& G, const lm_events& ev, const uint16_t* mu, const float* tof_tab,
               const TravLayout& L, char* base, cudaStream_t st);
// variant: the lane-group width 8, 16 or 32 (32 compiled for 3 resident
// blocks per SM), or 33 (width 32 compiled for 4 blocks per SM)
int launch_table_update(const TabArgs& a, int variant, int grid, cudaStream_t st);
int table_grid(int variant);

// ---- image kernels (lm_image.cu) ----
void launch_transpose_to_yf(const lm_grid* g, const float* src, float* dst, cudaStream_t st);
void launch_add_yf_to_std(const lm_grid* g, float* img, float* yf_acc, cudaStream_t st);
void launch_fold_fixed(const lm_grid* g, float* img, unsigned long long* a_std, unsigned long long* a_yf,
                       const unsigned* maxbits, long long count, float stepmax, cudaStream_t st);

// Tensor maps of one state's images for the TMA-staged image passes
// (grids with nx, ny multiples of 4, nx >= 40, ny >= 36).
struct alignas(128) TmaMaps {
    CUtensorMap xh[2];     // x (std), box {40, 34, 1} around a 32 x 32 tile (halo -4..+4 in x, -1..+1 in y)
    CUtensorMap xt[2];     // x (std), box {32, 32, 1}
    CUtensorMap w[2];      // w, (nx, ny, nz, ndim), box {36, 33, 1, ndim}
    CUtensorMap T, z, zc;  // box {32, 32, 1}
    CUtensorMap acc_std;   // float z pairs (2nx, ny, nz), box {64, 32, 1}; u64 (nx, ny, nz) when deterministic
    CUtensorMap acc_yf;    // the same in the y-fastest layout (2ny, nx, nz) / (ny, nx, nz)
    CUtensorMap dtvd;      // directional TV: D = P (w+ - w), shape and box of w (unset without the field)
};
bool tma_capable(const lm_grid* g);
int encode_tma_maps(const lm_grid* g, float* const x[2], float* const w[2], int ndim, float* T, float* z, float* zc,
                    void* acc_std, void* acc_yf, bool det, float* dtvd, TmaMaps* out);

struct ImgArgs {
    int n[3];
    int ndim;
    int V;
    const uint16_t* seq;   // selection (device); nullptr: mode fixed by `mode`
    int u;
    int n_subsets;
    int mode;              // IP_INIT / IP_UPDATE
    // x
    const float* x_cur;    // std
    float* x_nxt_std;
    float* x_nxt_yf;
    float* x_keep;         // IP_INIT: copy of x0 (x "used by the last update")
    // z
    float* z;
    float* zc;
    int kahan;
    const float* T;
    const float* sens;     // IP_INIT
    // data accumulators
    float* acc_std;
    float* acc_yf;
    unsigned long long* acci_std;
    unsigned long long* acci_yf;
    int det;
    const unsigned* maxbits;
    const int64_t* sub_off;
    float stepmax;
    unsigned* maxbits_reset;  // cleared for the next update
    int slot0;                // update u uses scale slot (slot0 + u) & 1
    // prior
    const float* w_cur[2];
    float* w_nxt[2];
    const int* wpar;
    float inv_p_data;      // 1/p_k = 2n
    float inv_p_prior;     // 1/p_{n+1} = 2
    float s_prior;         // S_{n+1} = gamma rho / ||K|| (fused prior step)
    float beta;
    // batched epochs
    float* xbuf[2];
    float* xbuf_yf[2];
    int* wpar_w;
    int* wbase;
    // TMA-staged passes
    int acc_pairs;         // 1: float accumulators hold (j, j + nx*ny) pairs (see EvArgs)
    const TmaMaps* tm;     // device copy of the state's maps, or nullptr
    int xcur;              // index of x_cur among the two x buffers
    int zlen;              // z slices per work item
    unsigned* err;         // set when a bounded wait gave up
    const float* xi;       // directional TV field [ndim][V], or nullptr (TV)
    const float* dtv_d;    // directional TV: P (w+ - w) from the dual step, or nullptr (formed here)
    int skip_prior;        // 1: return at once when the update is a prior update
    int skip_data;         // 1: return at once when the update is a data update
};

struct BatchImgArgs {
    const ImgArgs* slots;  // [cap]
    const int* active;     // [cap]
    int cap;
    int u;
    int64_t tiles_per_slot;
};
void launch_image_batch(const BatchImgArgs& b, int grid, cudaStream_t st);
void launch_wpar_batch(const BatchImgArgs& b, int count, cudaStream_t st);
int image_batch_grid(const lm_grid* g, int cap);
int64_t image_tiles(const lm_grid* g);
enum { IP_INIT = 0, IP_UPDATE = 1 };
void launch_image_pass(const ImgArgs& a, cudaStream_t st);
void launch_image_tma(const ImgArgs& a, cudaStream_t st);
void launch_image_tma_batch(const BatchImgArgs& b, int grid, cudaStream_t st);
int image_tma_batch_grid(const lm_grid* g, int cap);
int tma_zlen(const lm_grid* g);                       // z slices per TMA work item
int64_t tma_items_host(const lm_grid* g, int zlen);   // TMA work items of one image
void launch_wpar(const uint16_t* seq, int count, int n_subsets, int* wpar, int* wbase, cudaStream_t st);
void launch_step_T(const lm_grid* g, const float* sens, float* T, float rho, float gamma, double knorm, int n_subsets,
                   cudaStream_t st);
int reduce_minmax(const float* x, int64_t n, float* dev_scratch, float* mn, float* mx, cudaStream_t st);
void launch_zadd(const lm_grid* g, const float* z, const float* zc, float* out, cudaStream_t st);
// Image-space resolution model G (separable Gaussian, mirrored faces).
constexpr int RES_MAX_R = 31;  // taps per side
struct ResAxis {
    int r;
    float w[2 * RES_MAX_R + 1];  // w[k + r], k = -r..r
};
struct ResPlan {
    int n_axes;       // 0: G is the identity
    int axis[3];
    ResAxis ax[3];
};
int res_plan(const lm_grid* g, float fwhm, ResPlan& p);
// dst = G src via temporaries t1, t2; skipped when seq[u] >= n_subsets (seq set);
// pair_out: dst is a pair accumulator (values go to the first halves, the
// second halves are left zero); dst_yf: also the y-fastest copy of dst (or NULL)
int launch_res(const lm_grid* g, const ResPlan& p, const float* src, float* dst, float* t1, float* t2,
               const uint16_t* seq, int u, int n_subsets, cudaStream_t st, bool pair_out, float* dst_yf);
// G applied to the float pair accumulators (std and y-fastest) folded into
// one image; the result goes to the first halves of the std pairs and every
// other half is left zero.  s1, s2: V-float scratch images.
int launch_res_back(const lm_grid* g, const ResPlan& p, float* acc_std, float* acc_yf, float* s1, float* s2,
                    const uint16_t* seq, int u, int n_subsets, cudaStream_t st);
// out = the float pair accumulators (std and y-fastest) folded into one image; clears them
void launch_res_fold(const lm_grid* g, float* acc_std, float* acc_yf, float* out, const uint16_t* seq, int u,
                     int n_subsets, cudaStream_t st);

// out4: <sens, x>, ||Kx||_{2,1}, sum_e w_e log(p_e + s_e) (w = 1 if NULL), sum_e s_e if w is set (else 0);
// s_e = contam[e], or s_flat where contam is NULL
int objective_parts(const lm_grid* g, const float* sens, const float* x, const float* xi, const float* p,
                    const float* contam, float s_flat, const uint16_t* w, int64_t n_ev, double* scratch,
                    double* out4, cudaStream_t st);
size_t objective_scratch_bytes();

}  // namespace lmh
