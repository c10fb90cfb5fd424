// LM-SPDHG state and iteration (Alg. 2).
//
// Device memory is one caller-owned buffer, carved here.  Per update u the
// library launches two kernels (three in deterministic mode):
//   1. the event kernel: if the selection is a data subset, the fused
//      forward projection / dual step / back-projection of its events into
//      the dz accumulators; if it is the prior, the dual step of w;
//   2. the image pass: dz (accumulators, or K^T(w+ - w) for the prior) into
//      z with compensated summation, zbar = z + dz/p_i and the next primal
//      step x <- proj_{>=0}(x - T zbar), written in both image layouts.
// The selection is read on the device, so a whole epoch (2n updates) is one
// captured CUDA graph that serves every selection sequence.  x, w and the
// fixed-point scale slots alternate between two buffers; the w parity of
// each update is a prefix count of prior selections computed on the device.
#include <cmath>
#include <cstring>
#include <vector>

#include "lm_internal.h"

using namespace lmh;

struct lm_state_s {
    lm_scanner sc;
    lm_grid g;
    lm_tof tof;
    lmk::Geo G;
    lm_params P;
    int64_t N;
    int n;
    int ndim;
    int64_t V;
    bool two_d, det, kahan;
    double gamma, knorm;
    // caller arrays
    const int32_t *det1, *det2;
    const int16_t* tofb;
    const float *corr, *contam;
    const uint16_t* mu;
    const float* sens;
    std::vector<int64_t> sub_off_h;
    // carved device memory
    float *x[2], *xyf[2], *z, *zc, *T, *acc_std, *acc_yf, *w[2], *y, *scr;
    unsigned long long *acci_std, *acci_yf, *queue;
    int64_t* sub_off;
    uint16_t* seq;
    int* wpar;
    int* wbase;
    unsigned* maxbits;
    unsigned* done;
    float* redf;
    double* redd;
    float* tof_tab;   // tabulated TOF kernel (TOF_TAB_N + 1 floats)
    TmaMaps* tmaps;   // device copy of the tensor maps (TMA-staged image passes)
    unsigned* err;    // set by a bounded device wait that gave up
    bool tma;         // image passes staged by TMA (grid permitting, unless disabled)
    bool tma_data;    // TMA-staged data passes, plain prior passes (image_kernel 3)
    bool has_res;     // resolution model P = A G: the event kernels read G x from gx / gxyf
    float *gx, *gxyf; // G x in both layouts (float mode; scratch of the back-projection's G)
    float* rt;        // scratch image of the resolution model's passes (float mode)
    float* dtvd;      // directional TV: P (w+ - w) of the last prior dual step [ndim][V]
    ResPlan res;
    int zlen;         // z slices per TMA work item
    bool table;       // data updates from the traversal table (lm_table.cu)
    TravLayout tv;    // its layout in the caller's buffer
    char* tv_base;
    bool tiled;       // data updates by the tile-binned projector
    TileArgs ta;      // its per-frame tables (pointers into the caller's tile buffer)
    TileLayout tl;
    char* tile_base;
    int64_t n_segments;
    size_t scr_bytes;
    int grid_ev, grid_fx, chunk;
    int grid_tab;       // blocks of the traversal-table kernel
    int tab_variant;    // its compiled variant (launch_table_update)
    bool tab_split;     // one launch per principal-axis family (else one for all)
    int group;          // lanes per event of the event kernels
    double tune_ms[3];  // autotuner: forward projection of subset 0 with 8, 16, 32 lanes
    double tune_table_ms, tune_direct_ms;  // data update of subset 0: best table / direct variant
    cudaStream_t cap_stream;
    cudaGraphExec_t exec;
    bool have_graph;
    int64_t graph_nodes;
    bool persist;       // epochs in one persistent cooperative launch (2D float TV frames)
    int grid_persist;   // its blocks (all resident)
    unsigned* bar;      // its grid barrier: arrival count, generation
    const unsigned* gate;  // failure injection: a flag its first block waits for
    bool shard;         // event sharding: updates through lmspdhg_shard_begin / _finish
    float* dz;          // the exchange buffer: this state's partial back-projection [V]
    int shard_stage;    // 0 ready, 1 initialisation awaiting the exchange, 2 update awaiting it
    int shard_sel;      // selection of the update in progress
    int xpar;           // buffer holding the x the next update starts from
    int64_t n_updates;
};

namespace {

struct Carve {
    size_t off = 0;
    char* base = nullptr;
    template <class T>
    T* take(size_t bytes)
    {
        T* p = base ? (T*)(base + off) : nullptr;
        off += align_up(bytes);
        return p;
    }
};

void carve(lm_state* st, Carve& c, const lm_grid* g, int64_t N, int n, bool det, bool dtv, bool shard)
{
    const size_t V = (size_t)nvox(g);
    const int nd = std::max(1, tv_ndim(g));
    const bool yf = g->n[1] > 1;
    auto F = [&](size_t cnt) { return c.take<float>(cnt * 4); };
    float* x0 = F(V);
    float* x1 = F(V);
    float* y0 = yf ? F(V) : nullptr;
    float* y1 = yf ? F(V) : nullptr;
    float* z = F(V);
    float* zc = F(V);
    float* T = F(V);
    float* w0 = F(nd * V);
    float* w1 = F(nd * V);
    // float accumulators hold (voxel j, voxel j + nx*ny) pairs (scatter_pairs)
    float* acc_std = det ? nullptr : F(2 * V);
    float* acc_yf = (!det && yf) ? F(2 * V) : nullptr;
    unsigned long long* ai_std = det ? c.take<unsigned long long>(V * 8) : nullptr;
    unsigned long long* ai_yf = (det && yf) ? c.take<unsigned long long>(V * 8) : nullptr;
    // G x for the resolution model, both layouts (8 B per voxel, float mode)
    float* gx = det ? nullptr : F(V);
    float* gxyf = det ? nullptr : F(V);
    float* rt = det ? nullptr : F(V);
    float* dtvd = dtv ? F(nd * V) : nullptr;
    float* dz = shard ? F(V) : nullptr;
    float* y = F((size_t)std::max<int64_t>(N, 1));
    const size_t scr_bytes = std::max<size_t>((size_t)std::max<int64_t>(N, 1) * 4,
                                              std::max(lm_knorm_workspace_bytes(g), objective_scratch_bytes()));
    float* scr = c.take<float>(scr_bytes);
    int64_t* sub_off = c.take<int64_t>((size_t)(n + 1) * 8);
    uint16_t* seq = c.take<uint16_t>((size_t)2 * n * 2 + 64);
    int* wpar = c.take<int>((size_t)(2 * n + 2) * 4);
    int* wbase = c.take<int>(16);
    unsigned* maxbits = c.take<unsigned>(16);
    unsigned long long* queue = c.take<unsigned long long>(16);
    unsigned* done = c.take<unsigned>(16);
    float* redf = c.take<float>((2 * 1024 + 16) * 4);
    double* redd = c.take<double>(objective_scratch_bytes());
    float* tof_tab = c.take<float>((size_t)(TOF_TAB_N + 1) * 4);
    TmaMaps* tmaps = c.take<TmaMaps>(sizeof(TmaMaps));
    unsigned* err = c.take<unsigned>(16);
    unsigned* bar = c.take<unsigned>(16);
    if (st) {
        st->bar = bar;
        st->tof_tab = tof_tab;
        st->tmaps = tmaps;
        st->err = err;
        st->x[0] = x0; st->x[1] = x1; st->xyf[0] = y0; st->xyf[1] = y1;
        st->z = z; st->zc = zc; st->T = T; st->w[0] = w0; st->w[1] = w1;
        st->acc_std = acc_std; st->acc_yf = acc_yf; st->acci_std = ai_std; st->acci_yf = ai_yf;
        st->y = y; st->scr = scr; st->scr_bytes = scr_bytes; st->sub_off = sub_off; st->seq = seq;
        st->wpar = wpar; st->wbase = wbase; st->maxbits = maxbits; st->queue = queue; st->done = done;
        st->redf = redf; st->redd = redd;
        st->gx = gx; st->gxyf = gxyf; st->rt = rt; st->dtvd = dtvd; st->dz = dz;
    }
}

// The TMA-staged prior pass computes the prior's dual step itself (with the
// directional TV's field read where it needs it); the plain prior pass
// takes it from the event kernel's prior branch (which stores D = P (w+ - w)
// for the directional TV).
bool tma_fuses_prior(const lm_state* st) { return st->tma; }

EvArgs base_ev_args(const lm_state* st)
{
    EvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.G = st->G;
    a.det1 = st->det1;
    a.det2 = st->det2;
    a.tof = st->tofb;
    a.corr = st->corr;
    a.contam = st->contam;
    a.mu = st->mu;
    a.y = st->y;
    a.sub_off = st->sub_off;
    a.n_subsets = st->n;
    a.gamma_rho = (float)(st->gamma * (double)st->P.rho);
    a.stepmax = 2.0f * std::fmax(st->g.h[0], std::fmax(st->g.h[1], st->g.h[2]));
    a.queue = st->queue;
    a.done = st->done;
    a.chunk = st->chunk;
    a.w_cur[0] = st->w[0];
    a.w_cur[1] = st->w[1];
    a.w_nxt[0] = st->w[1];
    a.w_nxt[1] = st->w[0];
    a.wpar = st->wpar;
    a.s_prior = (float)(st->gamma * (double)st->P.rho / st->knorm);
    a.beta = st->P.beta;
    a.ndim = st->ndim;
    a.tof_tab = st->tof.n_bins > 0 ? st->tof_tab : nullptr;
    a.group = st->group;
    a.prior_fused = tma_fuses_prior(st) ? 1 : 0;
    a.acc_pairs = st->det ? 0 : 1;
    a.xi = st->P.xi;
    a.dtv_d = st->dtvd;
    a.sino = st->P.sinogram;
    if (st->P.sinogram == 2) {
        a.g_q = st->P.sino_q;
        a.g_qoff = st->P.sino_qoff;
        a.g_lorf = st->P.sino_lorf;
        a.g_s = st->P.sino_s;
        a.g_rings = st->sc.n_rings;
        a.g_xtal = st->sc.n_xtal;
        a.g_nb = std::max(1, (int)st->tof.n_bins);
    }
    return a;
}

ImgArgs base_img_args(const lm_state* st)
{
    ImgArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; ++d) a.n[d] = st->g.n[d];
    a.ndim = st->ndim;
    a.V = (int)st->V;
    a.n_subsets = st->n;
    a.z = st->z;
    a.zc = st->zc;
    a.kahan = st->kahan ? 1 : 0;
    a.T = st->T;
    a.sens = st->sens;
    a.acc_std = st->acc_std;
    a.acc_yf = st->acc_yf;
    a.acci_std = st->acci_std;
    a.acci_yf = st->acci_yf;
    a.det = st->det ? 1 : 0;
    a.maxbits = st->maxbits;
    a.maxbits_reset = st->maxbits;
    a.sub_off = st->sub_off;
    a.stepmax = 2.0f * std::fmax(st->g.h[0], std::fmax(st->g.h[1], st->g.h[2]));
    a.w_cur[0] = st->w[0];
    a.w_cur[1] = st->w[1];
    a.w_nxt[0] = st->w[1];
    a.w_nxt[1] = st->w[0];
    a.wpar = st->wpar;
    a.inv_p_data = (float)(2 * st->n);
    a.inv_p_prior = 2.0f;
    a.s_prior = (float)(st->gamma * (double)st->P.rho / st->knorm);
    a.beta = st->P.beta;
    a.acc_pairs = st->det ? 0 : 1;
    a.tm = (st->tma || st->tma_data) ? st->tmaps : nullptr;
    a.err = st->err;
    a.zlen = st->zlen;
    a.xi = st->P.xi;
    a.dtv_d = st->dtvd;
    return a;
}

// Arguments of the traversal-table data update of update u (x in buffer cur).
TabArgs base_tab_args(const lm_state* st, int cur)
{
    TabArgs t;
    std::memset(&t, 0, sizeof(t));
    t.G = st->G;
    t.r0 = (const float4*)(st->tv_base + st->tv.r0);
    t.r1 = (const float4*)(st->tv_base + st->tv.r1);
    t.meta = (const int2*)(st->tv_base + st->tv.meta);
    t.corr = st->corr;
    t.contam = st->contam;
    t.mu = st->mu;
    t.y = st->y;
    t.x_std = st->x[cur];
    t.x_yf = st->xyf[cur];
    t.acc_std = st->acc_std;
    t.acc_yf = st->acc_yf;
    t.tof_tab = st->tof_tab;
    t.sub_off = st->sub_off;
    t.n_subsets = st->n;
    t.gamma_rho = (float)(st->gamma * (double)st->P.rho);
    t.queue = st->queue;
    t.done = st->done;
    t.phase = -1;
    return t;
}

// Stores every event's traversal and (P^LM 1)_e in the caller's table buffer.
int build_table(lm_state* st, cudaStream_t s)
{
    lm_events ev;
    std::memset(&ev, 0, sizeof(ev));
    ev.det1 = st->det1;
    ev.det2 = st->det2;
    ev.tof = st->tofb;
    ev.corr = st->corr;
    ev.contam = st->contam;
    ev.n = st->N;
    return trav_build(st->G, ev, st->mu, st->tof_tab, st->tv, st->tv_base, s);
}

// Resolution model: G x into gx (x-fastest) and gxyf (y-fastest), through the
// scratch image rt (gxyf is the second scratch of the unfused passes, written
// last by the y-fastest copy).
int res_fwd(lm_state* st, const float* x, cudaStream_t s)
{
    return launch_res(&st->g, st->res, x, st->gx, st->rt, st->gxyf, nullptr, 0, 0, s, false,
                      st->g.n[1] > 1 ? st->gxyf : nullptr);
}

// Resolution model: G (A^T v) from the accumulators, written back as the
// first halves of the std pairs (every other half zero), so the image pass
// merges G A^T v unchanged.  G x is no longer needed by this update, so gx
// serves as scratch.  Skipped on the device when seq[u] selects the prior.
int res_back(lm_state* st, const uint16_t* seq, int u, cudaStream_t s)
{
    return launch_res_back(&st->g, st->res, st->acc_std, st->acc_yf, st->rt, st->gx, seq, u, st->n, s);
}

// The event part of update u (selection st->seq[u], x in buffer cur, scale
// slot `slot`): the data update's event kernels, which leave the
// back-projection of the dual change in the accumulators (or, with the
// directional TV or the plain image passes, the prior's dual step).
int launch_event_part(lm_state* st, int u, int cur, int slot, cudaStream_t s)
{
    EvArgs a = base_ev_args(st);
    a.seq = st->seq;
    a.u = u;
    a.x_std = st->has_res ? st->gx : st->x[cur];  // G x with the resolution model
    a.x_yf = st->has_res ? st->gxyf : st->xyf[cur];
    a.px = st->x[cur];
    a.maxbits = st->maxbits + slot;
    if (st->tiled) {
        TileArgs t = st->ta;
        t.seq = st->seq;
        t.u = u;
        t.x = st->x[cur];
        t.acc = st->acc_std;
        t.v = st->scr;
        t.gamma_rho = (float)(st->gamma * (double)st->P.rho);
        int rc = launch_tile_update(t, st->two_d, s);
        LM_CHECK(rc == LM_OK, rc, "tile data update launch failed");
        if (!tma_fuses_prior(st)) {
            // the image pass needs w+ (and D) from the event kernel's prior branch
            a.prior_only = 1;
            rc = launch_events(EV_DATA, st->two_d, a, st->grid_ev, s);
            LM_CHECK(rc == LM_OK, rc, "prior update launch failed");
        }
    } else if (st->table) {
        // the table kernel, one launch per principal-axis family so that one
        // image layout and one accumulator layout share L2 (both return at
        // once on a prior update)
        TabArgs t = base_tab_args(st, cur);
        t.seq = st->seq;
        t.u = u;
        int rc = LM_OK;
        for (int ph = st->tab_split ? 0 : -1; ph < (st->tab_split ? 2 : 0) && rc == LM_OK; ++ph) {
            t.phase = ph;
            rc = launch_table_update(t, st->tab_variant, st->grid_tab, s);
        }
        LM_CHECK(rc == LM_OK, rc, "data update launch failed");
        if (!tma_fuses_prior(st)) {
            // the image pass needs w+ (and D) from the event kernel's prior branch
            a.prior_only = 1;
            rc = launch_events(EV_DATA, st->two_d, a, st->grid_ev, s);
            LM_CHECK(rc == LM_OK, rc, "prior update launch failed");
        }
    } else if (!st->det) {
        a.acc_std = st->acc_std;
        a.acc_yf = st->acc_yf;
        int rc = launch_events(EV_DATA, st->two_d, a, st->grid_ev, s);
        LM_CHECK(rc == LM_OK, rc, "data update launch failed");
        if (st->has_res) {
            rc = res_back(st, st->seq, u, s);
            if (rc) return rc;
        }
    } else {
        a.out = st->scr;
        int rc = launch_events(EV_DATA_FX1, st->two_d, a, st->grid_ev, s);
        LM_CHECK(rc == LM_OK, rc, "data update launch failed");
        EvArgs b = base_ev_args(st);
        b.seq = st->seq;
        b.u = u;
        b.vin = st->scr;
        b.acci_std = st->acci_std;
        b.acci_yf = st->acci_yf;
        b.maxbits = st->maxbits + slot;
        rc = launch_events(EV_BACK_FX, st->two_d, b, st->grid_fx, s);
        LM_CHECK(rc == LM_OK, rc, "fixed-point back-projection launch failed");
    }
    return LM_OK;
}

// The image part of update u: merges the accumulators into z and z-bar (or
// runs the prior's steps) and takes the next primal step into buffer nxt.
int launch_image_part(lm_state* st, int u, int cur, int nxt, int slot0, cudaStream_t s)
{
    ImgArgs im = base_img_args(st);
    im.mode = IP_UPDATE;
    im.seq = st->seq;
    im.u = u;
    im.x_cur = st->x[cur];
    im.x_nxt_std = st->x[nxt];
    im.x_nxt_yf = st->xyf[nxt];
    // scale slots: update u reads slot (slot0 + u) & 1, its pass clears the other one
    im.slot0 = slot0;
    im.xcur = cur;
    if (st->tma) {
        launch_image_tma(im, s);
    } else if (st->tma_data) {
        // TMA-staged data passes, plain prior passes
        ImgArgs d = im, q = im;
        d.skip_prior = 1;
        q.skip_data = 1;
        launch_image_tma(d, s);
        launch_image_pass(q, s);
    } else {
        launch_image_pass(im, s);
    }
    if (st->has_res) {
        int rc = res_fwd(st, st->x[nxt], s);  // the next update's projections read G x
        if (rc) return rc;
    }
    return LM_OK;
}

// Launches updates 0..count-1 of the selection already in st->seq; x starts
// in buffer xpar0; the fixed-point scale slot of update u is (slot0 + u) & 1.
// If `ev` is given (profiling), events ev[3u], ev[3u+1], ev[3u+2] are
// recorded before the event kernel, before the image pass and after it.
int launch_updates(lm_state* st, int count, int xpar0, int slot0, cudaStream_t s, cudaEvent_t* ev = nullptr)
{
    launch_wpar(st->seq, count, st->n, st->wpar, st->wbase, s);
    for (int u = 0; u < count; ++u) {
        const int cur = (xpar0 + u) & 1, nxt = cur ^ 1;
        const int slot = (slot0 + u) & 1;
        if (ev) LM_CUDA(cudaEventRecord(ev[3 * u], s));
        int rc = launch_event_part(st, u, cur, slot, s);
        if (rc) return rc;
        if (ev) LM_CUDA(cudaEventRecord(ev[3 * u + 1], s));
        rc = launch_image_part(st, u, cur, nxt, slot0, s);
        if (rc) return rc;
        if (ev) LM_CUDA(cudaEventRecord(ev[3 * u + 2], s));
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// Initialisation of Alg. 2 and the first primal step for the state's current events:
// gamma, T, y = Eq. (yinit), z = P^T 1 + (P^LM)^T((y-1)/mu), w = 0, x from x0.
int chunk_for(int64_t count, int grid);

// The initialisation's image pass: z = P^T 1 + the accumulated
// back-projection, z-bar = z, T and the first primal step from x0; x0 is
// also kept in x[1] (the x the most recent update used).
int init_image_pass(lm_state* st, const float* x0, cudaStream_t s)
{
    ImgArgs im = base_img_args(st);
    im.mode = IP_INIT;
    im.x_cur = x0;
    im.x_keep = st->x[1];
    im.x_nxt_std = st->x[0];
    im.x_nxt_yf = st->xyf[0];
    launch_image_pass(im, s);
    if (st->has_res) {
        int rc = res_fwd(st, st->x[0], s);
        if (rc) return rc;
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// Event sharding: dz (summed over the states) back into the first halves of
// the z-paired accumulators, where the image passes read a data update's
// back-projection (the fold left both accumulators zero).
__global__ void unfold_pairs_kernel(const float* __restrict__ dz, float2* __restrict__ acc_std, int64_t V)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < V; j += (int64_t)gridDim.x * blockDim.x)
        acc_std[j] = make_float2(dz[j], 0.0f);
}

void launch_unfold(lm_state* st, cudaStream_t s)
{
    const int grid = (int)std::min<int64_t>((st->V + 255) / 256, (int64_t)num_sms() * 8);
    unfold_pairs_kernel<<<std::max(grid, 1), 256, 0, s>>>(st->dz, (float2*)st->acc_std, st->V);
    count_launch();
}

int init_iteration(lm_state* st, const float* x0, cudaStream_t s)
{
    const size_t V = (size_t)st->V;
    const bool yf = st->g.n[1] > 1;
    LM_CUDA(cudaMemsetAsync(st->zc, 0, V * 4, s));
    LM_CUDA(cudaMemsetAsync(st->w[0], 0, (size_t)std::max(1, st->ndim) * V * 4, s));
    LM_CUDA(cudaMemsetAsync(st->w[1], 0, (size_t)std::max(1, st->ndim) * V * 4, s));
    if (st->acc_std) LM_CUDA(cudaMemsetAsync(st->acc_std, 0, 2 * V * 4, s));
    if (st->acc_yf) LM_CUDA(cudaMemsetAsync(st->acc_yf, 0, 2 * V * 4, s));
    if (st->acci_std) LM_CUDA(cudaMemsetAsync(st->acci_std, 0, V * 8, s));
    if (st->acci_yf) LM_CUDA(cudaMemsetAsync(st->acci_yf, 0, V * 8, s));
    LM_CUDA(cudaMemsetAsync(st->wbase, 0, 16, s));
    LM_CUDA(cudaMemsetAsync(st->maxbits, 0, 16, s));
    LM_CUDA(cudaMemsetAsync(st->queue, 0, 16, s));
    LM_CUDA(cudaMemsetAsync(st->done, 0, 16, s));
    // x0 >= 0 and gamma = 3 / ||x0||_inf (Sec. "Numerical experiments")
    float mn = 0.0f, mx = 0.0f;
    int rc = reduce_minmax(x0, st->V, st->redf, &mn, &mx, s);
    if (rc) return rc;
    LM_CHECK(mn >= 0.0f, LM_ERR_DOMAIN, "x0 must be >= 0 (min %g)", (double)mn);
    if (st->P.gamma > 0.0f) {
        st->gamma = st->P.gamma;
    } else {
        LM_CHECK(mx > 0.0f, LM_ERR_DOMAIN, "gamma = 3/max(x0) needs max(x0) > 0");
        st->gamma = 3.0 / (double)mx;
    }
    launch_step_T(&st->g, st->sens, st->T, st->P.rho, (float)st->gamma, st->knorm, st->n, s);
    EvArgs a = base_ev_args(st);
    a.x_std = x0;
    if (st->has_res) {
        rc = res_fwd(st, x0, s);
        if (rc) return rc;
        a.x_std = st->gx;
        a.x_yf = yf ? st->gxyf : nullptr;
    } else if (yf) {
        launch_transpose_to_yf(&st->g, x0, st->xyf[1], s);
        a.x_yf = st->xyf[1];
    }
    a.e_begin = 0;
    a.e_end = st->N;
    a.chunk = chunk_for(st->N, st->grid_ev);  // all N events, not one subset
    if (st->N > 0) {
        if (!st->det) {
            a.acc_std = st->acc_std;
            a.acc_yf = st->acc_yf;
            rc = launch_events(EV_YINIT, st->two_d, a, st->grid_ev, s);
            if (!rc && st->has_res) rc = res_back(st, nullptr, 0, s);
        } else {
            a.out = st->scr;
            a.maxbits = st->maxbits + 1;
            rc = launch_events(EV_YINIT_FX1, st->two_d, a, st->grid_ev, s);
            if (!rc) {
                EvArgs b = base_ev_args(st);
                b.e_begin = 0;
                b.e_end = st->N;
                b.chunk = chunk_for(st->N, st->grid_fx);
                b.vin = st->scr;
                b.acci_std = st->acci_std;
                b.acci_yf = st->acci_yf;
                b.maxbits = st->maxbits + 1;
                rc = launch_events(EV_BACK_FX, st->two_d, b, st->grid_fx, s);
            }
        }
        LM_CHECK(rc == LM_OK, rc, "initialisation launch failed");
    }
    st->xpar = 0;
    st->n_updates = 0;
    if (st->shard) {
        // this state's part of the initialisation's back-projection goes to the exchange
        // buffer; z, T and the first primal step follow the caller's sum over the states
        // (lmspdhg_shard_init_finish), from the copy of x0 kept in x[1]
        launch_res_fold(&st->g, st->acc_std, st->acc_yf, st->dz, nullptr, 0, st->n, s);
        LM_CUDA(cudaMemcpyAsync(st->x[1], x0, V * 4, cudaMemcpyDeviceToDevice, s));
        LM_CUDA(cudaGetLastError());
        st->shard_stage = 1;
        return LM_OK;
    }
    return init_image_pass(st, x0, s);
}

// Autotuner: times the forward projection of subset 0 (x of the first
// update, both layouts) with 8, 16 and 32 lanes per event and keeps the
// fastest width.  Output goes to the per-event scratch; state is unchanged.
int autotune_group(lm_state* st, cudaStream_t s)
{
    st->tune_ms[0] = st->tune_ms[1] = st->tune_ms[2] = 0.0;
    const int64_t n0 = st->sub_off_h[1] - st->sub_off_h[0];
    if (n0 <= 0) return LM_OK;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    const int widths[3] = {8, 16, 32};
    double best = 1e30;
    int best_g = 16;
    for (int w = 0; w < 3; ++w) {
        EvArgs a = base_ev_args(st);
        a.group = widths[w];
        a.x_std = st->x[0];
        a.x_yf = st->xyf[0];
        a.out = st->scr;
        a.e_begin = st->sub_off_h[0];
        a.e_end = st->sub_off_h[1];
        a.queue = nullptr;
        a.done = nullptr;
        float tot = 0.0f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            int rc = launch_events(EV_FWD, st->two_d, a, ev_grid_g(EV_FWD, st->two_d, widths[w]), s);
            cudaEventRecord(e1, s);
            if (rc) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rc;
            }
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;  // first run warms caches
        }
        st->tune_ms[w] = tot / 2.0;
        if (st->tune_ms[w] < best) {
            best = st->tune_ms[w];
            best_g = widths[w];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st->group = best_g;
    return LM_OK;
}

// Autotuner of the traversal-table path: times the data update of subset 0
// (from the x of the first update) with 8, 16 and 32 lanes per event, three
// runs each (the first warms the caches), restoring the subset's duals
// before every run; the accumulators are cleared afterwards, so the state is
// as it was.
int autotune_table(lm_state* st, cudaStream_t s)
{
    st->tune_ms[0] = st->tune_ms[1] = st->tune_ms[2] = 0.0;
    const int64_t b0 = st->sub_off_h[0], n0 = st->sub_off_h[1] - st->sub_off_h[0];
    if (n0 <= 0) return LM_OK;
    float* ysave = st->scr;  // the per-event scratch holds N floats
    LM_CUDA(cudaMemcpyAsync(ysave, st->y + b0, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s));
    TabArgs t = base_tab_args(st, st->xpar);
    t.e_begin = b0;
    t.e_end = b0 + n0;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    // variants: widths 8, 16, 32 (3 blocks per SM) and 32 (4 blocks per SM)
    const int variants[4] = {8, 16, 32, 33};
    double ms[4] = {0.0, 0.0, 0.0, 0.0};
    double best = 1e30;
    int best_v = 32, rc = LM_OK;
    for (int w = 0; w < 4 && rc == LM_OK; ++w) {
        float tot = 0.0f;
        for (int rep = 0; rep < 3 && rc == LM_OK; ++rep) {
            cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s);
            cudaEventRecord(e0, s);
            rc = launch_table_update(t, variants[w], table_grid(variants[w]), s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float m = 0.0f;
            cudaEventElapsedTime(&m, e0, e1);
            if (rep > 0) tot += m;
        }
        ms[w] = tot / 2.0;
        if (ms[w] < best) {
            best = ms[w];
            best_v = variants[w];
        }
    }
    // the chosen variant with the principal-axis families in one launch
    // instead of two
    double one = 0.0;
    t.phase = -1;
    for (int rep = 0; rep < 3 && rc == LM_OK; ++rep) {
        cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(e0, s);
        rc = launch_table_update(t, best_v, table_grid(best_v), s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float m = 0.0f;
        cudaEventElapsedTime(&m, e0, e1);
        if (rep > 0) one += m / 2.0;
    }
    double two = 0.0;
    for (int rep = 0; rep < 3 && rc == LM_OK; ++rep) {
        cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(e0, s);
        for (int ph = 0; ph < 2 && rc == LM_OK; ++ph) {
            t.phase = ph;
            rc = launch_table_update(t, best_v, table_grid(best_v), s);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float m = 0.0f;
        cudaEventElapsedTime(&m, e0, e1);
        if (rep > 0) two += m / 2.0;
    }
    st->tab_split = two <= one;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    st->tune_ms[0] = ms[0];
    st->tune_ms[1] = ms[1];
    st->tune_ms[2] = std::min(ms[2], ms[3]);
    LM_CUDA(cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s));
    LM_CUDA(cudaMemsetAsync(st->acc_std, 0, 2 * (size_t)st->V * 4, s));
    LM_CUDA(cudaMemsetAsync(st->acc_yf, 0, 2 * (size_t)st->V * 4, s));
    st->tab_variant = best_v;
    const int best_g = best_v == 33 ? 32 : best_v;
    st->group = best_g;
    // the direct event kernel on the same subset: the projector with the shorter data update stays
    // (unless the caller keeps the table)
    const double table_ms = std::min(one, two);
    double direct_ms = 1e30;
    int direct_g = 32;
    if (!st->P.trav_keep) {
        cudaEvent_t d0, d1;
        LM_CUDA(cudaEventCreate(&d0));
        LM_CUDA(cudaEventCreate(&d1));
        const int widths[3] = {8, 16, 32};
        for (int w = 0; w < 3 && rc == LM_OK; ++w) {
            EvArgs a = base_ev_args(st);
            a.group = widths[w];
            a.x_std = st->x[st->xpar];
            a.x_yf = st->xyf[st->xpar];
            a.acc_std = st->acc_std;
            a.acc_yf = st->acc_yf;
            a.e_begin = b0;
            a.e_end = b0 + n0;
            a.chunk = chunk_for(n0, ev_grid_g(EV_DATA, st->two_d, widths[w]));
            double tot = 0.0;
            for (int rep = 0; rep < 3 && rc == LM_OK; ++rep) {
                cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s);
                cudaEventRecord(d0, s);
                rc = launch_events(EV_DATA, st->two_d, a, ev_grid_g(EV_DATA, st->two_d, widths[w]), s);
                cudaEventRecord(d1, s);
                cudaEventSynchronize(d1);
                float m = 0.0f;
                cudaEventElapsedTime(&m, d0, d1);
                if (rep > 0) tot += m / 2.0;
            }
            if (tot < direct_ms) {
                direct_ms = tot;
                direct_g = widths[w];
            }
        }
        cudaEventDestroy(d0);
        cudaEventDestroy(d1);
        if (rc) return rc;
        LM_CUDA(cudaMemcpyAsync(st->y + b0, ysave, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s));
        LM_CUDA(cudaMemsetAsync(st->acc_std, 0, 2 * (size_t)st->V * 4, s));
        LM_CUDA(cudaMemsetAsync(st->acc_yf, 0, 2 * (size_t)st->V * 4, s));
    }
    st->tune_table_ms = table_ms;
    st->tune_direct_ms = st->P.trav_keep ? 0.0 : direct_ms;
    if (!st->P.trav_keep && direct_ms < table_ms) {
        st->table = false;
        st->group = direct_g;
    }
    return LM_OK;
}

// Events per work item for a launch over `count` events on `grid` blocks of
// 8 warps: about four items per warp, between 1 and 32 (a whole warp's
// per-lane set-up).
int chunk_for(int64_t count, int grid)
{
    const int64_t ch = count / std::max<int64_t>(1, (int64_t)grid * 8 * 4);
    return (int)std::max<int64_t>(1, std::min<int64_t>(32, ch));
}

int choose_chunk(const lm_state* st)
{
    int64_t maxsub = 0;
    for (int k = 0; k < st->n; ++k) maxsub = std::max<int64_t>(maxsub, st->sub_off_h[k + 1] - st->sub_off_h[k]);
    const int64_t warps = (int64_t)st->grid_ev * 8;
    int64_t ch = maxsub / std::max<int64_t>(1, warps * 4);
    return (int)std::max<int64_t>(1, std::min<int64_t>(32, ch));
}

}  // namespace

extern "C" {

size_t lmspdhg_tile_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets)
{
    if (check_grid(grid) || n_events < 0 || n_subsets < 1) return 0;
    return tile_layout(grid, n_events, n_subsets).total;
}

size_t lmspdhg_trav_bytes(const lm_grid* grid, int64_t n_events)
{
    if (check_grid(grid) || n_events < 0 || !trav_capable(grid)) return 0;
    return trav_layout(grid, n_events).total;
}

size_t lmspdhg_state_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets, int32_t deterministic)
{
    if (check_grid(grid) || n_events < 0 || n_subsets < 1) return 0;
    Carve c;
    carve(nullptr, c, grid, n_events, n_subsets, deterministic != 0, false, false);
    return c.off + 256;
}

size_t lmspdhg_state_bytes_ex(const lm_grid* grid, int64_t n_events, int32_t n_subsets, const lm_params* params)
{
    if (check_grid(grid) || n_events < 0 || n_subsets < 1 || params == nullptr) return 0;
    Carve c;
    carve(nullptr, c, grid, n_events, n_subsets, params->deterministic != 0, params->xi != nullptr,
          params->shard != 0);
    return c.off + 256;
}

int lmspdhg_create(lm_state** out, const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                   const lm_events* ev, const uint16_t* mu, const int64_t* sub_off_host, const float* sens,
                   const float* x0, const lm_params* params, void* state_buf, size_t state_bytes, void* stream)
{
    clear_error();
    LM_CHECK(out != nullptr && params != nullptr && ev != nullptr, LM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    lmk::Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    const lm_params& P = *params;
    LM_CHECK(P.n_subsets >= 1 && P.n_subsets < 65535, LM_ERR_INVALID_ARG, "n_subsets out of range");
    LM_CHECK(P.beta >= 0.0f && std::isfinite(P.beta), LM_ERR_INVALID_ARG, "beta must be >= 0");
    LM_CHECK(P.rho > 0.0f && std::isfinite(P.rho), LM_ERR_INVALID_ARG, "rho must be > 0");
    LM_CHECK(P.sinogram >= 0 && P.sinogram <= 2, LM_ERR_INVALID_ARG, "sinogram must be 0, 1 or 2");
    if (P.sinogram == 2) {
        LM_CHECK(ev->n == lm_sino_n_bins(sc, tof) && mu && P.sino_q && P.sino_qoff, LM_ERR_INVALID_ARG,
                 "a generated sinogram needs every bin's count and the subsets' pair lists");
        LM_CHECK(P.sino_s > 0.0f && std::isfinite(P.sino_s), LM_ERR_DOMAIN, "sino_s must be > 0");
    } else {
        LM_CHECK(ev->n >= 0 && (ev->n == 0 || (ev->det1 && ev->det2 && ev->contam && mu)), LM_ERR_INVALID_ARG,
                 "events need det1, det2, contam and mu");
        LM_CHECK(tof->n_bins == 0 || ev->n == 0 || ev->tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL");
    }
    LM_CHECK(sens && x0 && sub_off_host && state_buf, LM_ERR_INVALID_ARG, "NULL sens, x0, sub_off or state buffer");
    LM_CHECK(sub_off_host[0] == 0 && sub_off_host[P.n_subsets] == ev->n, LM_ERR_INVALID_ARG,
             "subset offsets must span [0, n)");
    for (int k = 0; k < P.n_subsets; ++k)
        LM_CHECK(sub_off_host[k + 1] >= sub_off_host[k], LM_ERR_INVALID_ARG, "subset offsets must not decrease");
    LM_CHECK(P.image_kernel >= 0 && P.image_kernel <= 3, LM_ERR_INVALID_ARG, "image_kernel must be 0, 1, 2 or 3");
    LM_CHECK(!(P.image_kernel == 2 || P.image_kernel == 3) || tma_capable(grid), LM_ERR_INVALID_ARG,
             "the TMA-staged image pass needs nx, ny multiples of 4 with nx >= 40, ny >= 36");
    LM_CHECK(P.res_fwhm >= 0.0f, LM_ERR_INVALID_ARG, "res_fwhm must be >= 0");
    if (P.res_fwhm > 0.0f) {
        LM_CHECK(P.deterministic == 0, LM_ERR_INVALID_ARG, "the resolution model runs in float-atomic mode");
        ResPlan rp;
        rc = res_plan(grid, P.res_fwhm, rp);
        if (rc) return rc;
    }
    LM_CHECK(P.shard == 0 || P.shard == 1, LM_ERR_INVALID_ARG, "shard must be 0 or 1");
    LM_CHECK(P.epoch_kernel >= 0 && P.epoch_kernel <= 2, LM_ERR_INVALID_ARG, "epoch_kernel must be 0, 1 or 2");
    LM_CHECK(!P.shard || (!P.deterministic && P.res_fwhm == 0.0f && !P.sinogram && P.tile_buf == nullptr),
             LM_ERR_INVALID_ARG,
             "event sharding runs in float-atomic mode without the resolution model, sinogram bins or tiles");
    const size_t need = lmspdhg_state_bytes_ex(grid, ev->n, P.n_subsets, &P);
    LM_CHECK(state_bytes >= need, LM_ERR_NOMEM, "state buffer needs %zu bytes", need);

    lm_state* st = new lm_state();
    st->sc = *sc;
    st->g = *grid;
    st->tof = *tof;
    st->G = G;
    st->P = P;
    st->N = ev->n;
    st->n = P.n_subsets;
    st->ndim = tv_ndim(grid);
    st->V = nvox(grid);
    st->two_d = grid->n[2] == 1 && sc->n_rings == 1;
    st->det = P.deterministic != 0;
    st->kahan = P.kahan != 0;
    st->shard = P.shard != 0;
    st->shard_stage = 0;
    st->shard_sel = 0;
    st->det1 = ev->det1;
    st->det2 = ev->det2;
    st->tofb = ev->tof;
    st->corr = ev->corr;
    st->contam = ev->contam;
    st->mu = mu;
    st->sens = sens;
    st->sub_off_h.assign(sub_off_host, sub_off_host + P.n_subsets + 1);
    Carve c;
    c.base = (char*)(((uintptr_t)state_buf + 255) / 256 * 256);
    carve(st, c, grid, ev->n, st->n, st->det, P.xi != nullptr, P.shard != 0);
    st->exec = nullptr;
    st->have_graph = false;
    st->xpar = 0;
    st->n_updates = 0;
    if (cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete st;
        set_error("cudaStreamCreate failed");
        return LM_ERR_CUDA;
    }
    auto fail = [&](int code) {
        cudaStreamDestroy(st->cap_stream);
        delete st;
        return code;
    };
    cudaStream_t s = S(stream);
#define LM_TRY(call)                                                                    \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_error("%s: %s", #call, cudaGetErrorString(e_));                         \
            return fail(LM_ERR_CUDA);                                                   \
        }                                                                               \
    } while (0)
    LM_TRY(cudaMemcpyAsync(st->sub_off, sub_off_host, (size_t)(st->n + 1) * 8, cudaMemcpyHostToDevice, s));
    LM_TRY(cudaMemsetAsync(st->err, 0, 16, s));
    st->tma = false;
    st->tma_data = false;
    st->zlen = 1;
    st->has_res = P.res_fwhm > 0.0f;
    if (st->has_res) res_plan(grid, P.res_fwhm, st->res);  // validated above
    if (P.image_kernel != 1 && tma_capable(grid)) {
        TmaMaps h;
        rc = encode_tma_maps(grid, st->x, st->w, std::max(1, st->ndim), st->T, st->z, st->zc,
                             st->det ? (void*)st->acci_std : (void*)st->acc_std,
                             st->det ? (void*)st->acci_yf : (void*)st->acc_yf, st->det, st->dtvd, &h);
        if (rc) return fail(rc);
        LM_TRY(cudaMemcpyAsync(st->tmaps, &h, sizeof(h), cudaMemcpyHostToDevice, s));
        LM_TRY(cudaStreamSynchronize(s));
        st->tma = P.image_kernel != 3;
        st->tma_data = P.image_kernel == 3;
        st->zlen = tma_zlen(grid);
    }
    if (tof->n_bins > 0) {
        std::vector<float> tab(TOF_TAB_N + 1);
        tof_table(tof, tab.data());
        LM_TRY(cudaMemcpyAsync(st->tof_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s));
        LM_TRY(cudaStreamSynchronize(s));
    }
    st->tiled = false;
    st->n_segments = 0;
    st->tile_base = nullptr;
    st->tune_table_ms = 0.0;
    st->tune_direct_ms = 0.0;
    if (P.tile_buf != nullptr && tof->n_bins > 0 && !st->det && !st->has_res && !P.sinogram && grid->n[0] < 16384 && grid->n[1] < 16384 &&
        grid->n[2] < 16384) {
        st->tl = tile_layout(grid, ev->n, st->n);
        if (P.tile_bytes < st->tl.total) {
            set_error("tile buffer of %zu bytes, %zu needed", P.tile_bytes, st->tl.total);
            return fail(LM_ERR_NOMEM);
        }
        char* tb = (char*)(((uintptr_t)P.tile_buf + 255) / 256 * 256);
        if (P.tile_bytes - (size_t)(tb - (char*)P.tile_buf) < st->tl.total - 256) {
            set_error("tile buffer too small after alignment");
            return fail(LM_ERR_NOMEM);
        }
        st->tile_base = tb;
        TileArgs& t = st->ta;
        std::memset(&t, 0, sizeof(t));
        t.G = st->G;
        tile_geometry(grid, t.ntile, &t.tz, &t.n_tiles);
        t.n_subsets = st->n;
        t.tof_tab = st->tof_tab;
        t.det1 = st->det1;
        t.det2 = st->det2;
        t.tofb = st->tofb;
        t.corr = st->corr;
        t.contam = st->contam;
        t.mu = st->mu;
        t.y = st->y;
        t.sub_off = st->sub_off;
        t.evp = (float4*)(tb + st->tl.evp);
        t.p1 = (float*)(tb + st->tl.p1);
        t.seg_off = (unsigned*)(tb + st->tl.seg_off);
        t.seg = (uint2*)(tb + st->tl.seg);
        t.seg_pos = (unsigned*)(tb + st->tl.seg_pos);
        t.part = (float*)(tb + st->tl.part);
        t.items = (TileItem*)(tb + st->tl.items);
        t.item_off = (int*)(tb + st->tl.item_off);
        tile_attributes();
        rc = tile_build(t, st->tl, tb, ev->n, st->sub_off_h, st->two_d, s, &st->n_segments);
        if (rc == LM_ERR_NOMEM) {
            clear_error();  // more segments than the buffer holds: the direct kernel serves this frame
            st->n_segments = 0;
        } else if (rc) {
            return fail(rc);
        } else {
            st->tiled = true;
        }
    }
    st->table = false;
    st->tv_base = nullptr;
    if (P.trav_buf != nullptr && tof->n_bins > 0 && !st->det && !st->has_res && !P.sinogram && !st->tiled &&
        trav_capable(grid)) {
        st->tv = trav_layout(grid, ev->n);
        char* tb = (char*)(((uintptr_t)P.trav_buf + 255) / 256 * 256);
        if (P.trav_bytes < st->tv.total || P.trav_bytes - (size_t)(tb - (char*)P.trav_buf) < st->tv.total - 256) {
            set_error("traversal-table buffer of %zu bytes, %zu needed", P.trav_bytes, st->tv.total);
            return fail(LM_ERR_NOMEM);
        }
        st->tv_base = tb;
        rc = build_table(st, s);
        if (rc) return fail(rc);
        st->table = true;
    }
    if (P.knorm > 0.0) {
        st->knorm = P.knorm;
    } else if (st->ndim == 0) {
        st->knorm = 1.0;
    } else {
        double kn = 0.0;
        rc = lm_knorm_fp64(grid, P.knorm_iters > 0 ? P.knorm_iters : 1000, st->scr, st->scr_bytes, &kn, stream);
        if (rc) return fail(rc);
        st->knorm = kn;
    }
    st->grid_ev = ev_grid(st->det ? EV_DATA_FX1 : EV_DATA, st->two_d);
    st->grid_fx = ev_grid(EV_BACK_FX, st->two_d);
    st->chunk = choose_chunk(st);
    st->group = (P.group == 8 || P.group == 16 || P.group == 32) ? P.group : 16;
    rc = init_iteration(st, x0, s);
    if (rc) return fail(rc);
    if (P.group == 0) {
        rc = st->table ? autotune_table(st, s) : autotune_group(st, s);
        if (rc) return fail(rc);
    }
    if (P.group != 0) {
        st->tab_variant = st->group;
        st->tab_split = true;
    }
    st->gate = nullptr;
    {
        const bool fits = st->two_d && !st->det && !st->has_res && !P.sinogram && !st->tiled && !st->table &&
                          P.xi == nullptr && !st->shard && persist_supported() && persist_grid(st->group) > 0;
        if (P.epoch_kernel == 2 && !fits) {
            set_error("the persistent epoch kernel serves 2D float-mode TV frames with the direct projector");
            return fail(LM_ERR_INVALID_ARG);
        }
        // measured on the 2D frame: the captured graph of per-update launches is faster (its 2n
        // updates need 4n grid barriers in one launch), so auto keeps the graph
        st->persist = fits && P.epoch_kernel == 2;
        st->grid_persist = st->persist ? persist_grid(st->group) : 0;
    }
    st->grid_tab = st->table ? table_grid(st->tab_variant) : 0;
    // the event kernels run with as many resident blocks as the chosen width allows
    st->grid_ev = ev_grid_g(st->det ? EV_DATA_FX1 : EV_DATA, st->two_d, st->group);
    st->grid_fx = ev_grid_g(EV_BACK_FX, st->two_d, st->group);
    st->chunk = choose_chunk(st);
    LM_TRY(cudaStreamSynchronize(s));
#undef LM_TRY
    *out = st;
    return LM_OK;
}

int lmspdhg_updates(lm_state* st, const uint16_t* seq_host, int32_t count, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    LM_CHECK(!st->shard, LM_ERR_INVALID_ARG, "a shard state updates through lmspdhg_shard_begin / _finish");
    LM_CHECK(count >= 0, LM_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return LM_OK;
    LM_CHECK(seq_host != nullptr, LM_ERR_INVALID_ARG, "seq is NULL");
    for (int i = 0; i < count; ++i)
        LM_CHECK(seq_host[i] <= st->n, LM_ERR_INVALID_ARG, "selection %d out of range", (int)seq_host[i]);
    cudaStream_t s = S(stream);
    const int chunk = 2 * st->n;
    for (int b = 0; b < count; b += chunk) {
        const int m = std::min(chunk, count - b);
        LM_CUDA(cudaMemcpyAsync(st->seq, seq_host + b, (size_t)m * 2, cudaMemcpyHostToDevice, s));
        int rc = launch_updates(st, m, st->xpar, (int)(st->n_updates & 1), s);
        if (rc) return rc;
        st->xpar ^= (m & 1);
        st->n_updates += m;
    }
    return LM_OK;
}

int lmspdhg_epoch(lm_state* st, const uint16_t* seq_host, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr && seq_host != nullptr, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(!st->shard, LM_ERR_INVALID_ARG, "a shard state updates through lmspdhg_shard_begin / _finish");
    const int count = 2 * st->n;
    for (int i = 0; i < count; ++i)
        LM_CHECK(seq_host[i] <= st->n, LM_ERR_INVALID_ARG, "selection %d out of range", (int)seq_host[i]);
    cudaStream_t s = S(stream);
    if (st->persist) {
        LM_CUDA(cudaMemcpyAsync(st->seq, seq_host, (size_t)count * 2, cudaMemcpyHostToDevice, s));
        launch_wpar(st->seq, count, st->n, st->wpar, st->wbase, s);
        LM_CUDA(cudaMemsetAsync(st->bar, 0, 16, s));
        PersistArgs p;
        std::memset(&p, 0, sizeof(p));
        p.ev = base_ev_args(st);
        p.ev.acc_std = st->acc_std;
        p.ev.acc_yf = st->acc_yf;
        p.ev.queue = nullptr;
        p.ev.done = nullptr;
        for (int b = 0; b < 2; ++b) {
            p.xs[b] = st->x[b];
            p.xw[b] = st->x[b];
            p.xyf[b] = st->xyf[b];
        }
        p.seq = st->seq;
        p.count = count;
        p.xpar0 = st->xpar;
        p.z = st->z;
        p.zc = st->zc;
        p.T = st->T;
        p.kahan = st->kahan ? 1 : 0;
        p.inv_p_data = (float)(2 * st->n);
        p.inv_p_prior = 2.0f;
        p.bar = st->bar;
        p.err = st->err;
        p.gate = st->gate;
        int rc = launch_persist_epoch(p, st->group, st->grid_persist, s);
        if (rc) return rc;
        st->xpar ^= (count & 1);
        st->n_updates += count;
        return LM_OK;
    }
    if (st->xpar != 0 || (st->n_updates & 1)) return lmspdhg_updates(st, seq_host, count, stream);
    if (!st->have_graph) {
        cudaGraph_t graph = nullptr;
        LM_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = launch_total();
        int rc = launch_updates(st, count, 0, 0, st->cap_stream);
        st->graph_nodes = launch_total() - before;
        count_launch(-st->graph_nodes);  // captured, not run
        cudaError_t ce = cudaStreamEndCapture(st->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&st->exec, graph, 0);
        cudaGraphDestroy(graph);
        LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
        st->have_graph = true;
    }
    LM_CUDA(cudaMemcpyAsync(st->seq, seq_host, (size_t)count * 2, cudaMemcpyHostToDevice, s));
    LM_CUDA(cudaGraphLaunch(st->exec, s));
    count_launch(st->graph_nodes);
    st->n_updates += count;
    return LM_OK;
}

int lmspdhg_reinit(lm_state* st, const float* x0, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr && x0 != nullptr, LM_ERR_INVALID_ARG, "NULL argument");
    if (st->tiled) {
        // the events may be another frame's: bin them again
        int rc = tile_build(st->ta, st->tl, st->tile_base, st->N, st->sub_off_h, st->two_d, S(stream),
                            &st->n_segments);
        if (rc == LM_ERR_NOMEM) {
            clear_error();  // this frame needs more segments than the buffer holds: direct kernel
            st->tiled = false;
            st->n_segments = 0;
        } else if (rc) {
            return rc;
        }
    }
    LM_CUDA(cudaMemsetAsync(st->err, 0, 16, S(stream)));  // a fresh start clears a wait that gave up
    if (st->table) {
        // the events may be another frame's: store their traversals again
        int rc = build_table(st, S(stream));
        if (rc) return rc;
    }
    return init_iteration(st, x0, S(stream));
}

int lmspdhg_projector(lm_state* st, int32_t* kind, int64_t* n_segments)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    if (kind) *kind = st->table ? 3 : (st->tiled ? 2 : 1);
    if (n_segments) *n_segments = st->tiled ? st->n_segments : 0;
    return LM_OK;
}

int lmspdhg_profile(lm_state* st, const uint16_t* seq_host, int32_t count, double* ms4, int64_t* n4,
                    void* stream)
{
    clear_error();
    LM_CHECK(st && seq_host && ms4 && n4, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(!st->shard, LM_ERR_INVALID_ARG, "a shard state updates through lmspdhg_shard_begin / _finish");
    LM_CHECK(count >= 1 && count <= 2 * st->n, LM_ERR_INVALID_ARG, "count must be in [1, 2n]");
    for (int i = 0; i < count; ++i)
        LM_CHECK(seq_host[i] <= st->n, LM_ERR_INVALID_ARG, "selection %d out of range", (int)seq_host[i]);
    cudaStream_t s = S(stream);
    std::vector<cudaEvent_t> ev((size_t)3 * count);
    for (auto& e : ev) LM_CUDA(cudaEventCreate(&e));
    LM_CUDA(cudaMemcpyAsync(st->seq, seq_host, (size_t)count * 2, cudaMemcpyHostToDevice, s));
    int rc = launch_updates(st, count, st->xpar, (int)(st->n_updates & 1), s, ev.data());
    if (rc == LM_OK) {
        st->xpar ^= (count & 1);
        st->n_updates += count;
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = LM_ERR_CUDA;
    }
    for (int k = 0; k < 4; ++k) {
        ms4[k] = 0.0;
        n4[k] = 0;
    }
    if (rc == LM_OK) {
        for (int u = 0; u < count; ++u) {
            const int prior = seq_host[u] >= st->n;
            float t1 = 0.0f, t2 = 0.0f;
            cudaEventElapsedTime(&t1, ev[3 * u], ev[3 * u + 1]);
            cudaEventElapsedTime(&t2, ev[3 * u + 1], ev[3 * u + 2]);
            ms4[prior] += t1;
            n4[prior] += 1;
            ms4[2 + prior] += t2;
            n4[2 + prior] += 1;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (rc == LM_ERR_CUDA) set_error("profiling run failed");
    return rc;
}

int lmspdhg_get_x(lm_state* st, float* x_out, void* stream)
{
    clear_error();
    LM_CHECK(st && x_out, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CUDA(cudaMemcpyAsync(x_out, st->x[st->xpar ^ 1], (size_t)st->V * 4, cudaMemcpyDeviceToDevice, S(stream)));
    return LM_OK;
}

int lmspdhg_get_y(lm_state* st, float* y_out, void* stream)
{
    clear_error();
    LM_CHECK(st && y_out, LM_ERR_INVALID_ARG, "NULL argument");
    if (st->N == 0) return LM_OK;
    LM_CUDA(cudaMemcpyAsync(y_out, st->y, (size_t)st->N * 4, cudaMemcpyDeviceToDevice, S(stream)));
    return LM_OK;
}

int lmspdhg_get_z(lm_state* st, float* z_out, void* stream)
{
    clear_error();
    LM_CHECK(st && z_out, LM_ERR_INVALID_ARG, "NULL argument");
    launch_zadd(&st->g, st->z, st->kahan ? st->zc : nullptr, z_out, S(stream));
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

int lmspdhg_get_w(lm_state* st, float* w_out, void* stream)
{
    clear_error();
    LM_CHECK(st && w_out, LM_ERR_INVALID_ARG, "NULL argument");
    if (st->ndim == 0) return LM_OK;
    // the current w buffer is given by the device-side parity base
    int wb = 0;
    LM_CUDA(cudaMemcpyAsync(&wb, st->wbase, 4, cudaMemcpyDeviceToHost, S(stream)));
    LM_CUDA(cudaStreamSynchronize(S(stream)));
    LM_CUDA(cudaMemcpyAsync(w_out, st->w[wb & 1], (size_t)st->ndim * st->V * 4, cudaMemcpyDeviceToDevice,
                            S(stream)));
    return LM_OK;
}

int lmspdhg_objective_fp64(lm_state* st, double* out_host, void* stream)
{
    clear_error();
    LM_CHECK(st && out_host, LM_ERR_INVALID_ARG, "NULL argument");
    double parts[4];
    int rc = lmspdhg_objective_parts_fp64(st, parts, stream);
    if (rc) return rc;
    // listmode: <P^T 1, x> - sum_e log(...) + beta R (Eq. (1) without the constant sum of s);
    // sinogram bins: Eq. (1) itself, sum_b (Px + s)_b - d_b log(Px + s)_b + beta R
    *out_host = parts[0] - parts[2] + (double)st->P.beta * parts[1] + parts[3];
    return LM_OK;
}

int lmspdhg_objective_parts_fp64(lm_state* st, double* out4, void* stream)
{
    clear_error();
    LM_CHECK(st && out4, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(st->shard_stage == 0, LM_ERR_INVALID_ARG, "an exchange of the shard protocol is pending");
    cudaStream_t s = S(stream);
    const int xb = st->xpar ^ 1;
    float* p = st->scr;
    if (st->N > 0) {
        EvArgs a = base_ev_args(st);
        a.x_std = st->x[xb];
        a.x_yf = st->xyf[xb];
        if (st->has_res) {
            // G x into the (zero) accumulators, which the next update does not read before clearing
            float* t = st->acc_std;
            int rc = launch_res(&st->g, st->res, st->x[xb], t, t + st->V, st->acc_yf ? st->acc_yf : t + st->V,
                                nullptr, 0, 0, s, false, nullptr);
            if (rc) return rc;
            a.x_std = t;
            a.x_yf = nullptr;
        }
        a.out = p;
        a.e_begin = 0;
        a.e_end = st->N;
        a.queue = nullptr;
        a.done = nullptr;
        a.chunk = 32;
        int rc = launch_events(EV_FWD, st->two_d, a, ev_grid_g(EV_FWD, st->two_d, st->group), s);
        LM_CHECK(rc == LM_OK, rc, "objective projection failed");
        if (st->has_res) {
            // the accumulators must be zero at the next update
            LM_CUDA(cudaMemsetAsync(st->acc_std, 0, 2 * (size_t)st->V * 4, s));
            if (st->acc_yf) LM_CUDA(cudaMemsetAsync(st->acc_yf, 0, 2 * (size_t)st->V * 4, s));
        }
    }
    int rc = objective_parts(&st->g, st->sens, st->x[xb], st->P.xi, p, st->contam, st->P.sino_s,
                             st->P.sinogram ? st->mu : nullptr, st->N, st->redd, out4, s);
    if (rc) return rc;
    unsigned err = 0;
    LM_CUDA(cudaMemcpyAsync(&err, st->err, sizeof(err), cudaMemcpyDeviceToHost, s));
    LM_CUDA(cudaStreamSynchronize(s));
    LM_CHECK(err == 0, LM_ERR_TIMEOUT, "a bounded wait of the image pass gave up; the iterate is not valid");
    return LM_OK;
}

int lmspdhg_shard_buffer(lm_state* st, float** dz_out)
{
    clear_error();
    LM_CHECK(st && dz_out, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(st->shard, LM_ERR_INVALID_ARG, "not a shard state (lm_params.shard)");
    *dz_out = st->dz;
    return LM_OK;
}

int lmspdhg_shard_init_finish(lm_state* st, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    LM_CHECK(st->shard && st->shard_stage == 1, LM_ERR_INVALID_ARG,
             "no initialisation awaits its exchange (shard state after create / reinit)");
    cudaStream_t s = S(stream);
    launch_unfold(st, s);
    int rc = init_image_pass(st, st->x[1], s);
    if (rc) return rc;
    st->shard_stage = 0;
    return LM_OK;
}

int lmspdhg_shard_begin(lm_state* st, uint16_t sel, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    LM_CHECK(st->shard && st->shard_stage == 0, LM_ERR_INVALID_ARG,
             "a shard update starts after the initialisation's or the previous update's finish");
    LM_CHECK(sel <= st->n, LM_ERR_INVALID_ARG, "selection %d out of range", (int)sel);
    cudaStream_t s = S(stream);
    const uint16_t h = sel;
    LM_CUDA(cudaMemcpyAsync(st->seq, &h, 2, cudaMemcpyHostToDevice, s));
    LM_CUDA(cudaStreamSynchronize(s));  // h lives on this stack frame
    launch_wpar(st->seq, 1, st->n, st->wpar, st->wbase, s);
    int rc = launch_event_part(st, 0, st->xpar, (int)(st->n_updates & 1), s);
    if (rc) return rc;
    if (sel < st->n) launch_res_fold(&st->g, st->acc_std, st->acc_yf, st->dz, nullptr, 0, st->n, s);
    LM_CUDA(cudaGetLastError());
    st->shard_sel = sel;
    st->shard_stage = 2;
    return LM_OK;
}

int lmspdhg_shard_finish(lm_state* st, void* stream)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    LM_CHECK(st->shard && st->shard_stage == 2, LM_ERR_INVALID_ARG, "no shard update awaits its finish");
    cudaStream_t s = S(stream);
    if (st->shard_sel < st->n) launch_unfold(st, s);
    const int cur = st->xpar;
    int rc = launch_image_part(st, 0, cur, cur ^ 1, (int)(st->n_updates & 1), s);
    if (rc) return rc;
    LM_CUDA(cudaGetLastError());
    st->xpar ^= 1;
    st->n_updates += 1;
    st->shard_stage = 0;
    return LM_OK;
}

int lmspdhg_info(lm_state* st, int64_t* n_updates, double* gamma, double* knorm)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    if (n_updates) *n_updates = st->n_updates;
    if (gamma) *gamma = st->gamma;
    if (knorm) *knorm = st->knorm;
    return LM_OK;
}

int lmspdhg_image_kernel(lm_state* st, int32_t* kind)
{
    clear_error();
    LM_CHECK(st && kind, LM_ERR_INVALID_ARG, "NULL argument");
    *kind = st->tma ? 2 : (st->tma_data ? 3 : 1);
    return LM_OK;
}

int lmspdhg_tuning_projectors(lm_state* st, double* table_ms, double* direct_ms)
{
    clear_error();
    LM_CHECK(st && table_ms && direct_ms, LM_ERR_INVALID_ARG, "NULL argument");
    *table_ms = st->tune_table_ms;
    *direct_ms = st->tune_direct_ms;
    return LM_OK;
}

int lmspdhg_set_gate(lm_state* st, const unsigned* flag)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    st->gate = flag;
    return LM_OK;
}

int lmspdhg_epoch_kernel(lm_state* st, int32_t* kind)
{
    clear_error();
    LM_CHECK(st && kind, LM_ERR_INVALID_ARG, "NULL argument");
    *kind = st->persist ? 2 : 1;
    return LM_OK;
}

int lmspdhg_tuning(lm_state* st, int32_t* group, double* ms3)
{
    clear_error();
    LM_CHECK(st != nullptr, LM_ERR_INVALID_ARG, "state is NULL");
    if (group) *group = st->group;
    if (ms3)
        for (int k = 0; k < 3; ++k) ms3[k] = st->tune_ms[k];
    return LM_OK;
}

int lmspdhg_destroy(lm_state* st)
{
    clear_error();
    if (!st) return LM_OK;
    if (st->exec) cudaGraphExecDestroy(st->exec);
    cudaStreamDestroy(st->cap_stream);
    delete st;
    return LM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched epochs: several frames (states of the same scanner, grid, TOF
// kernel, subset count and mode) advance by one epoch in one captured graph
// whose kernels spread work over all occupied slots.  The per-slot argument
// tables live in a caller workspace; filling or emptying a slot rewrites its
// table entry only, so the same graph serves any occupancy and frames can
// join or leave between epochs.
// ---------------------------------------------------------------------------
// The configuration every state of a batch shares (copied from the first
// state set, which may be destroyed while the batch lives on).
struct BatchCfg {
    lm_grid g;
    lm_tof tof;
    float W;
    int n, n_det, group, zlen;
    bool two_d, det, kahan, tma;
    bool table;       // frames with traversal tables (the batch's data updates from them)
    int tab_variant;
};

struct lm_batch_s {
    int cap = 0;
    int n = 0;
    lm_state* slot[BATCH_MAX] = {};
    bool have_cfg = false;
    BatchCfg cfg;
    float* d_tof = nullptr;   // the batch's own copy of the TOF table
    EvArgs* d_ev = nullptr;
    ImgArgs* d_im = nullptr;
    TabArgs* d_tab = nullptr;
    int* d_active = nullptr;
    uint16_t* d_seqs = nullptr;
    unsigned long long* d_queue = nullptr;
    unsigned* d_done = nullptr;
    std::vector<EvArgs> h_ev;
    std::vector<ImgArgs> h_im;
    std::vector<TabArgs> h_tab;
    std::vector<int> h_active;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool have_graph = false;
    int64_t graph_nodes = 0;
};

namespace {

struct BatchLayout {
    size_t ev, im, tab, active, seqs, ctr, tof, total;
};

BatchLayout batch_layout(int cap, int n)
{
    BatchLayout L;
    size_t off = 0;
    L.ev = off;
    off += align_up(sizeof(EvArgs) * (size_t)cap);
    L.im = off;
    off += align_up(sizeof(ImgArgs) * (size_t)cap);
    L.tab = off;
    off += align_up(sizeof(TabArgs) * (size_t)cap);
    L.active = off;
    off += align_up(sizeof(int) * (size_t)cap);
    L.seqs = off;
    off += align_up(sizeof(uint16_t) * (size_t)cap * 2 * n);
    L.ctr = off;
    off += 256;
    L.tof = off;
    off += align_up((size_t)(TOF_TAB_N + 1) * 4);
    L.total = off + 256;
    return L;
}

BatchCfg cfg_of(const lm_state* st)
{
    BatchCfg c;
    c.g = st->g;
    c.tof = st->tof;
    c.W = st->G.W;
    c.n = st->n;
    c.n_det = st->G.n_det;
    c.group = st->group;
    c.zlen = st->zlen;
    c.two_d = st->two_d;
    c.det = st->det;
    c.kahan = st->kahan;
    c.tma = st->tma;
    c.table = st->table;
    c.tab_variant = st->tab_variant;
    return c;
}

bool same_config(const BatchCfg& a, const lm_state* st)
{
    const BatchCfg b = cfg_of(st);
    for (int d = 0; d < 3; ++d)
        if (a.g.n[d] != b.g.n[d]) return false;
    return a.n == b.n && a.two_d == b.two_d && a.det == b.det && a.kahan == b.kahan && a.tof.n_bins == b.tof.n_bins &&
           a.tof.sigma_mm == b.tof.sigma_mm && a.tof.bin_mm == b.tof.bin_mm && a.tof.n_sigma == b.tof.n_sigma &&
           a.n_det == b.n_det && a.group == b.group && a.tma == b.tma && a.zlen == b.zlen && a.table == b.table &&
           (!a.table || a.tab_variant == b.tab_variant);
}

void fill_slot(lm_batch* b, int s, lm_state* st)
{
    EvArgs a = base_ev_args(st);
    a.queue = nullptr;
    a.done = nullptr;
    // work items of a batched update span every frame: whole-warp chunks keep the
    // shared work counter's traffic low even when the frames are small
    a.chunk = 32;
    a.seq = b->d_seqs + (size_t)s * 2 * b->n;
    a.xb[0] = st->x[0];
    a.xb[1] = st->x[1];
    a.xbyf[0] = st->xyf[0];
    a.xbyf[1] = st->xyf[1];
    a.maxbits_base = st->maxbits;
    if (!st->det) {
        a.acc_std = st->acc_std;
        a.acc_yf = st->acc_yf;
    } else {
        a.acci_std = st->acci_std;
        a.acci_yf = st->acci_yf;
        a.out = st->scr;
        a.vin = st->scr;
    }
    ImgArgs im = base_img_args(st);
    im.mode = IP_UPDATE;
    im.seq = b->d_seqs + (size_t)s * 2 * b->n;
    im.slot0 = 0;
    im.xbuf[0] = st->x[0];
    im.xbuf[1] = st->x[1];
    im.xbuf_yf[0] = st->xyf[0];
    im.xbuf_yf[1] = st->xyf[1];
    im.wpar_w = st->wpar;
    im.wbase = st->wbase;
    b->h_ev[s] = a;
    b->h_im[s] = im;
    if (st->table) {
        TabArgs t = base_tab_args(st, 0);
        t.seq = nullptr;  // the batch reads the frames' selections itself
        t.queue = nullptr;
        t.done = nullptr;
        for (int k = 0; k < 2; ++k) {
            t.xs[k] = st->x[k];
            t.xyfs[k] = st->xyf[k];
        }
        b->h_tab[s] = t;
    }
}

int launch_batch_epoch(lm_batch* b, cudaStream_t s)
{
    const BatchCfg& r = b->cfg;
    const int count = 2 * b->n;
    BatchImgArgs bi;
    bi.slots = b->d_im;
    bi.active = b->d_active;
    bi.cap = b->cap;
    bi.u = 0;
    bi.tiles_per_slot = r.tma ? tma_items_host(&r.g, r.zlen) : image_tiles(&r.g);
    launch_wpar_batch(bi, count, s);
    BatchEvArgs be;
    std::memset(&be, 0, sizeof(be));
    be.slots = b->d_ev;
    be.active = b->d_active;
    be.seqs = b->d_seqs;
    be.seq_stride = count;
    be.cap = b->cap;
    be.slot0 = 0;
    be.queue = b->d_queue;
    be.done = (unsigned*)(b->d_queue + 1);
    be.tof_tab = r.tof.n_bins > 0 ? b->d_tof : nullptr;
    be.tof_W = r.W;
    be.vitem = 2048;
    BatchTabArgs bt;
    std::memset(&bt, 0, sizeof(bt));
    bt.slots = b->d_tab;
    bt.active = b->d_active;
    bt.seqs = b->d_seqs;
    bt.seq_stride = count;
    bt.cap = b->cap;
    bt.queue = b->d_queue;
    bt.done = (unsigned*)(b->d_queue + 1);
    bt.tof_tab = b->d_tof;
    bt.tof_W = r.W;
    const int g_tab = r.table ? table_grid(r.tab_variant) : 0;
    const int g_ev = ev_batch_grid(r.det ? EV_DATA_FX1 : EV_DATA, r.two_d, r.group);
    const int g_fx = ev_batch_grid(EV_BACK_FX, r.two_d, r.group);
    const int g_im = r.tma ? image_tma_batch_grid(&r.g, b->cap) : image_batch_grid(&r.g, b->cap);
    for (int u = 0; u < count; ++u) {
        be.u = u;
        bi.u = u;
        bt.u = u;
        int rc;
        if (r.table && r.tma) {
            // data updates from the frames' traversal tables (the prior's dual step is in the image pass)
            rc = launch_table_batch(bt, r.tab_variant, g_tab, s);
        } else if (!r.det) {
            rc = launch_events_batch(EV_DATA, r.two_d, r.group, be, g_ev, s);
        } else {
            rc = launch_events_batch(EV_DATA_FX1, r.two_d, r.group, be, g_ev, s);
            if (!rc) rc = launch_events_batch(EV_BACK_FX, r.two_d, r.group, be, g_fx, s);
        }
        LM_CHECK(rc == LM_OK, rc, "batched event kernel launch failed");
        if (r.tma) launch_image_tma_batch(bi, g_im, s);
        else launch_image_batch(bi, g_im, s);
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

}  // namespace

extern "C" {

size_t lmspdhg_batch_bytes(int32_t capacity, int32_t n_subsets)
{
    if (capacity < 1 || capacity > BATCH_MAX || n_subsets < 1) return 0;
    return batch_layout(capacity, n_subsets).total;
}

int lmspdhg_batch_create(lm_batch** out, int32_t capacity, int32_t n_subsets, void* buf, size_t bytes,
                         void* stream)
{
    clear_error();
    LM_CHECK(out != nullptr, LM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    LM_CHECK(capacity >= 1 && capacity <= BATCH_MAX, LM_ERR_INVALID_ARG, "capacity must be in [1, %d]", BATCH_MAX);
    LM_CHECK(n_subsets >= 1, LM_ERR_INVALID_ARG, "n_subsets must be >= 1");
    const BatchLayout L = batch_layout(capacity, n_subsets);
    LM_CHECK(buf != nullptr && bytes >= L.total, LM_ERR_NOMEM, "batch buffer needs %zu bytes", L.total);
    lm_batch* b = new lm_batch();
    b->cap = capacity;
    b->n = n_subsets;
    char* base = (char*)(((uintptr_t)buf + 255) / 256 * 256);
    b->d_ev = (EvArgs*)(base + L.ev);
    b->d_im = (ImgArgs*)(base + L.im);
    b->d_tab = (TabArgs*)(base + L.tab);
    b->d_active = (int*)(base + L.active);
    b->d_seqs = (uint16_t*)(base + L.seqs);
    b->d_queue = (unsigned long long*)(base + L.ctr);
    b->d_tof = (float*)(base + L.tof);
    b->h_ev.assign(capacity, EvArgs());
    b->h_im.assign(capacity, ImgArgs());
    b->h_tab.assign(capacity, TabArgs());
    b->h_active.assign(capacity, 0);
    cudaStream_t s = S(stream);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemsetAsync(base, 0, L.total - 256, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
        delete b;
        set_error("batch initialisation failed");
        return LM_ERR_CUDA;
    }
    *out = b;
    return LM_OK;
}

int lmspdhg_batch_set(lm_batch* b, int32_t slot, lm_state* st, void* stream)
{
    clear_error();
    LM_CHECK(b != nullptr && slot >= 0 && slot < b->cap, LM_ERR_INVALID_ARG, "bad batch or slot");
    cudaStream_t s = S(stream);
    if (st != nullptr) {
        LM_CHECK(st->n == b->n, LM_ERR_INVALID_ARG, "state has %d subsets, batch %d", st->n, b->n);
        LM_CHECK(!st->has_res, LM_ERR_INVALID_ARG, "states with the resolution model do not run in batches");
        LM_CHECK(!st->shard, LM_ERR_INVALID_ARG, "shard states do not run in batches");
        LM_CHECK(!b->have_cfg || same_config(b->cfg, st), LM_ERR_INVALID_ARG,
                 "state differs from the batch's grid, TOF kernel or mode");
        LM_CHECK(st->xpar == 0 && (st->n_updates & 1) == 0, LM_ERR_INVALID_ARG,
                 "a state joins a batch at an even update count");
        for (int k = 0; k < b->cap; ++k)
            LM_CHECK(k == slot || b->slot[k] != st, LM_ERR_INVALID_ARG, "state is already in slot %d", k);
        if (!b->have_cfg) {
            b->cfg = cfg_of(st);
            b->have_cfg = true;
            if (st->tof.n_bins > 0)
                LM_CUDA(cudaMemcpyAsync(b->d_tof, st->tof_tab, (size_t)(TOF_TAB_N + 1) * 4, cudaMemcpyDeviceToDevice,
                                        s));
        }
        fill_slot(b, slot, st);
        b->slot[slot] = st;
        b->h_active[slot] = 1;
        LM_CUDA(cudaMemcpyAsync(b->d_ev + slot, &b->h_ev[slot], sizeof(EvArgs), cudaMemcpyHostToDevice, s));
        LM_CUDA(cudaMemcpyAsync(b->d_im + slot, &b->h_im[slot], sizeof(ImgArgs), cudaMemcpyHostToDevice, s));
        if (st->table)
            LM_CUDA(cudaMemcpyAsync(b->d_tab + slot, &b->h_tab[slot], sizeof(TabArgs), cudaMemcpyHostToDevice, s));
    } else {
        b->slot[slot] = nullptr;
        b->h_active[slot] = 0;
    }
    LM_CUDA(cudaMemcpyAsync(b->d_active + slot, &b->h_active[slot], sizeof(int), cudaMemcpyHostToDevice, s));
    LM_CUDA(cudaStreamSynchronize(s));
    return LM_OK;
}

int lmspdhg_batch_epoch(lm_batch* b, const uint16_t* seqs_host, void* stream)
{
    clear_error();
    LM_CHECK(b != nullptr && seqs_host != nullptr, LM_ERR_INVALID_ARG, "NULL argument");
    const int count = 2 * b->n;
    int active = 0;
    for (int k = 0; k < b->cap; ++k) {
        if (!b->h_active[k]) continue;
        ++active;
        for (int u = 0; u < count; ++u)
            LM_CHECK(seqs_host[(size_t)k * count + u] <= b->n, LM_ERR_INVALID_ARG, "slot %d: selection out of range", k);
    }
    if (active == 0) return LM_OK;
    cudaStream_t s = S(stream);
    if (!b->have_graph) {
        cudaGraph_t graph = nullptr;
        LM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int64_t before = launch_total();
        int rc = launch_batch_epoch(b, b->cap_stream);
        b->graph_nodes = launch_total() - before;
        count_launch(-b->graph_nodes);
        cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "batch graph capture failed: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        LM_CHECK(ce == cudaSuccess, LM_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(ce));
        b->have_graph = true;
    }
    LM_CUDA(cudaMemcpyAsync(b->d_seqs, seqs_host, (size_t)b->cap * count * sizeof(uint16_t), cudaMemcpyHostToDevice,
                            s));
    LM_CUDA(cudaGraphLaunch(b->exec, s));
    count_launch(b->graph_nodes);
    for (int k = 0; k < b->cap; ++k)
        if (b->h_active[k]) b->slot[k]->n_updates += count;
    return LM_OK;
}

int lmspdhg_batch_destroy(lm_batch* b)
{
    clear_error();
    if (!b) return LM_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return LM_OK;
}

}  // extern "C"
