// Reconstruction server: continuous batching of LM-SPDHG frames.
//
// Frames (event lists with their selection sequences) are submitted from any
// host thread and queued.  A worker thread admits queued frames, in arrival
// order, into the slots of one lm_batch whenever a slot is free and the
// caller's device pool has room for the frame's events and state (first-fit
// allocation with coalescing free list); it then advances every admitted
// frame by one epoch in one batched graph launch, and retires frames that
// reached their epoch count (x and the objective copied to the host, memory
// released).  New frames therefore join while others are on the GPU.
// Callers wait for a ticket with a bounded timeout.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "lm_internal.h"

namespace {

__global__ void fill_kernel(float* x, int64_t n, float v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// First-fit allocator over [0, size) with coalescing of freed ranges.
class PoolAllocator {
public:
    explicit PoolAllocator(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off)
    {
        bytes = lmh::align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = lmh::align_up(bytes);
        used_ -= bytes;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

using Clock = std::chrono::steady_clock;

struct Frame {
    int64_t ticket = 0;
    int64_t n = 0;
    float x0 = 0.0f;
    std::vector<int32_t> det1, det2;
    std::vector<int16_t> tof;
    std::vector<float> corr, contam;
    std::vector<uint16_t> seqs;  // epochs * 2n
    Clock::time_point t_submit, t_done;
    // device resources while admitted
    size_t off = 0, bytes = 0;
    lm_state* st = nullptr;
    float* scratch = nullptr;  // V floats: x0 before create, free afterwards
    int slot = -1;
    int epochs_done = 0;
    // result
    bool done = false;
    int status = LM_OK;
    std::string error;
    std::vector<float> x;
    double objective = 0.0;
};

}  // namespace

struct lm_server_s {
    lm_scanner sc;
    lm_grid g;
    lm_tof tof;
    const float* sens = nullptr;
    lm_server_config cfg;
    char* pool = nullptr;
    PoolAllocator* alloc = nullptr;
    void* setup_ws = nullptr;  // shared event set-up workspace (front of the pool)
    size_t setup_ws_bytes = 0;
    lm_batch* batch = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;   // batched epochs and retirement
    cudaStream_t astream = nullptr;  // admission (uploads, event set-up, create), overlapping the epochs
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Frame*> queue;
    std::vector<Frame*> active;
    std::map<int64_t, Frame*> frames;
    int64_t next_ticket = 1;
    int64_t completed = 0;
    int64_t max_in_flight = 0;
    bool stop = false;
    std::thread worker;
};

namespace {

// Traversal-table bytes of a frame of n events (TOF data, 3D grid, float
// mode: the batch then runs its data updates from the tables), else 0.
size_t trav_bytes(const lm_server_s* s, int64_t n)
{
    if (s->tof.n_bins <= 0 || s->cfg.deterministic) return 0;
    return lmspdhg_trav_bytes(&s->g, n);
}

size_t frame_bytes(const lm_server_s* s, int64_t n)
{
    const size_t a = lmh::align_up((size_t)n * 4);
    const size_t h = lmh::align_up((size_t)n * 2);
    const size_t raw = 2 * a + h + 2 * a;             // det1, det2, tof, corr, contam
    const size_t perm = 2 * a + h + 2 * a + h;        // + mu
    const size_t x0 = lmh::align_up((size_t)lmh::nvox(&s->g) * 4);
    return raw + perm + x0 + lmh::align_up(trav_bytes(s, n)) +
           lmspdhg_state_bytes(&s->g, n, s->cfg.n_subsets, s->cfg.deterministic) + 512;
}

void fail_frame(lm_server_s* s, Frame* f, int code, const char* msg)
{
    f->status = code;
    f->error = msg;
    f->done = true;
    f->t_done = Clock::now();
    s->completed++;
}

// Admission of one frame: events uploaded into its pool range, set up, and
// its state created (on the admission stream, while the batch runs the
// current epoch on the other); joining the batch happens after the epoch.
// Called by the worker without the lock.
int prepare(lm_server_s* s, Frame* f)
{
    cudaStream_t st = s->astream;
    const int64_t n = f->n;
    char* base = s->pool + f->off;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* p = base + o;
        o += lmh::align_up(bytes);
        return p;
    };
    int32_t* r1 = (int32_t*)take(n * 4);
    int32_t* r2 = (int32_t*)take(n * 4);
    int16_t* rt = (int16_t*)take(n * 2);
    float* rc = (float*)take(n * 4);
    float* rs = (float*)take(n * 4);
    int32_t* p1 = (int32_t*)take(n * 4);
    int32_t* p2 = (int32_t*)take(n * 4);
    int16_t* pt = (int16_t*)take(n * 2);
    float* pc = (float*)take(n * 4);
    float* ps = (float*)take(n * 4);
    uint16_t* mu = (uint16_t*)take(n * 2);
    float* x0 = (float*)take((size_t)lmh::nvox(&s->g) * 4);
    const size_t tb = trav_bytes(s, n);
    char* trav = tb ? take(tb) : nullptr;
    char* stbuf = take(lmspdhg_state_bytes(&s->g, n, s->cfg.n_subsets, s->cfg.deterministic));
    const size_t stbytes = f->bytes - (size_t)(stbuf - base);
    LM_CUDA(cudaMemcpyAsync(r1, f->det1.data(), n * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(r2, f->det2.data(), n * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(rt, f->tof.data(), n * 2, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(rc, f->corr.data(), n * 4, cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaMemcpyAsync(rs, f->contam.data(), n * 4, cudaMemcpyHostToDevice, st));
    lm_events raw = {r1, r2, rt, rc, rs, n};
    std::vector<int64_t> off(s->cfg.n_subsets + 1);
    int rc0 = lm_event_setup(&s->sc, &s->tof, &raw, s->cfg.n_subsets, p1, p2, pt, pc, ps, mu, off.data(),
                             s->setup_ws, s->setup_ws_bytes, st);
    if (rc0) return rc0;
    const int64_t V = lmh::nvox(&s->g);
    fill_kernel<<<(int)std::min<int64_t>((V + 255) / 256, 4096), 256, 0, st>>>(x0, V, f->x0);
    lmh::count_launch();
    lm_events perm = {p1, p2, pt, pc, ps, n};
    lm_params P;
    std::memset(&P, 0, sizeof(P));
    P.beta = s->cfg.beta;
    P.rho = s->cfg.rho;
    P.knorm = s->cfg.knorm;
    P.n_subsets = s->cfg.n_subsets;
    P.deterministic = s->cfg.deterministic;
    P.kahan = s->cfg.kahan;
    P.group = s->cfg.group > 0 ? s->cfg.group : 32;
    P.trav_buf = trav;  // every frame of the batch keeps its traversals
    P.trav_keep = 1;
    P.trav_bytes = tb;
    lm_state* state = nullptr;
    rc0 = lmspdhg_create(&state, &s->sc, &s->g, &s->tof, &perm, mu, off.data(), s->sens, x0, &P, stbuf, stbytes,
                         st);
    if (rc0) return rc0;
    f->st = state;
    f->scratch = x0;
    // the host copies are no longer needed
    std::vector<int32_t>().swap(f->det1);
    std::vector<int32_t>().swap(f->det2);
    std::vector<int16_t>().swap(f->tof);
    std::vector<float>().swap(f->corr);
    std::vector<float>().swap(f->contam);
    return LM_OK;
}

int retire(lm_server_s* s, Frame* f)
{
    const int64_t V = lmh::nvox(&s->g);
    f->x.resize(V);
    int rc = lmspdhg_get_x(f->st, f->scratch, s->stream);  // lmspdhg_create copied x0
    if (!rc) {
        if (cudaMemcpyAsync(f->x.data(), f->scratch, V * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            rc = LM_ERR_CUDA;
    }
    if (!rc) rc = lmspdhg_objective_fp64(f->st, &f->objective, s->stream);
    lmspdhg_batch_set(s->batch, f->slot, nullptr, s->stream);
    lmspdhg_destroy(f->st);
    f->st = nullptr;
    f->slot = -1;
    return rc;
}

void finish_frame(lm_server_s* s, Frame* f, int rc, const char* what)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->alloc->release(f->off, f->bytes);
    if (rc) {
        fail_frame(s, f, rc, what);
    } else {
        f->done = true;
        f->t_done = Clock::now();
        s->completed++;
    }
}

// Worker loop: plan admissions; launch one batched epoch of the frames on
// the GPU; prepare the admitted frames meanwhile; wait for the epoch, retire
// the frames that are done and let the prepared ones join for the next
// epoch.
void worker_main(lm_server_s* s)
{
    cudaSetDevice(s->device);
    const int cap = s->cfg.max_slots;
    const int count = 2 * s->cfg.n_subsets;
    std::vector<uint16_t> seqs((size_t)cap * count);
    for (;;) {
        std::vector<Frame*> to_admit;
        std::vector<Frame*> act;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                                [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
            if (s->stop) break;
            // admission: FIFO, while a slot is free and the pool has room
            std::vector<bool> used(cap, false);
            for (Frame* f : s->active) used[f->slot] = true;
            int k = 0;
            while (!s->queue.empty()) {
                while (k < cap && used[k]) ++k;
                if (k == cap) break;
                Frame* f = s->queue.front();
                size_t off = 0;
                if (!s->alloc->alloc(f->bytes, &off)) break;  // wait for memory
                f->off = off;
                f->slot = k;
                used[k] = true;
                s->queue.pop_front();
                to_admit.push_back(f);
            }
            act = s->active;
        }
        int rc = LM_OK;
        if (!act.empty()) {
            std::fill(seqs.begin(), seqs.end(), (uint16_t)0);
            for (Frame* f : act)
                std::memcpy(&seqs[(size_t)f->slot * count], &f->seqs[(size_t)f->epochs_done * count], count * 2);
            rc = lmspdhg_batch_epoch(s->batch, seqs.data(), s->stream);
        }
        std::vector<Frame*> ready;
        for (Frame* f : to_admit) {
            const int r = prepare(s, f);
            if (r) {
                finish_frame(s, f, r, lm_last_error());
                s->cv_done.notify_all();
            } else {
                ready.push_back(f);
            }
        }
        if (!act.empty()) {
            if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = LM_ERR_CUDA;
            std::vector<Frame*> finished;
            for (Frame* f : act) {
                f->epochs_done++;
                if (rc || f->epochs_done >= s->cfg.epochs) finished.push_back(f);
            }
            for (Frame* f : finished) {
                const int r2 = rc ? rc : retire(s, f);
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->active.erase(std::find(s->active.begin(), s->active.end(), f));
                }
                finish_frame(s, f, r2, "epoch or retirement failed");
            }
            if (!finished.empty()) s->cv_done.notify_all();
        }
        for (Frame* f : ready) {
            const int r = lmspdhg_batch_set(s->batch, f->slot, f->st, s->stream);
            if (r) {
                lmspdhg_destroy(f->st);
                f->st = nullptr;
                finish_frame(s, f, r, "joining the batch failed");
                s->cv_done.notify_all();
                continue;
            }
            std::lock_guard<std::mutex> lk(s->mu);
            s->active.push_back(f);
            s->max_in_flight = std::max<int64_t>(s->max_in_flight, (int64_t)s->active.size());
        }
    }
}

}  // namespace

using namespace lmh;

extern "C" {

size_t lm_server_frame_bytes(const lm_grid* grid, int64_t n_events, int32_t n_subsets, int32_t deterministic)
{
    if (check_grid(grid) || n_events < 0 || n_subsets < 1) return 0;
    lm_server_s tmp;
    tmp.g = *grid;
    tmp.cfg.n_subsets = n_subsets;
    tmp.cfg.deterministic = deterministic;
    return frame_bytes(&tmp, n_events);
}

int lm_server_create(lm_server** out, const lm_scanner* sc, const lm_grid* grid, const lm_tof* tof,
                     const float* sens, const lm_server_config* cfg, void* pool, size_t pool_bytes)
{
    clear_error();
    LM_CHECK(out && sc && grid && tof && sens && cfg && pool, LM_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    lmk::Geo G;
    int rc = make_geo(sc, grid, tof, G, true);
    if (rc) return rc;
    LM_CHECK(cfg->max_slots >= 1 && cfg->max_slots <= BATCH_MAX, LM_ERR_INVALID_ARG, "max_slots in [1, %d]",
             BATCH_MAX);
    LM_CHECK(cfg->epochs >= 1 && cfg->n_subsets >= 1 && cfg->knorm > 0.0 && cfg->max_events >= 1,
             LM_ERR_INVALID_ARG, "epochs, n_subsets, knorm and max_events must be positive");
    lm_server_s* s = new lm_server_s();
    s->sc = *sc;
    s->g = *grid;
    s->tof = *tof;
    s->sens = sens;
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    char* base = (char*)(((uintptr_t)pool + 255) / 256 * 256);
    const size_t usable = pool_bytes - (size_t)(base - (char*)pool);
    s->setup_ws_bytes = lm_setup_workspace_bytes(cfg->max_events);
    const size_t bb = lmspdhg_batch_bytes(cfg->max_slots, cfg->n_subsets);
    const size_t head = align_up(s->setup_ws_bytes) + align_up(bb);
    if (usable < head + frame_bytes(s, cfg->max_events)) {
        delete s;
        set_error("pool of %zu bytes cannot hold the set-up workspace and one frame of max_events", pool_bytes);
        return LM_ERR_NOMEM;
    }
    s->setup_ws = base;
    void* bbuf = base + align_up(s->setup_ws_bytes);
    s->pool = base + head;
    s->alloc = new PoolAllocator(usable - head);
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->astream, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->stream) cudaStreamDestroy(s->stream);
        delete s->alloc;
        delete s;
        set_error("stream creation failed");
        return LM_ERR_CUDA;
    }
    rc = lmspdhg_batch_create(&s->batch, cfg->max_slots, cfg->n_subsets, bbuf, bb, s->stream);
    if (rc) {
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->astream);
        delete s->alloc;
        delete s;
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LM_OK;
}

int lm_server_submit(lm_server* s, const int32_t* det1, const int32_t* det2, const int16_t* tof, const float* corr,
                     const float* contam, int64_t n, float x0_value, const uint16_t* seqs_host,
                     int64_t* ticket)
{
    clear_error();
    LM_CHECK(s && det1 && det2 && contam && seqs_host && ticket, LM_ERR_INVALID_ARG, "NULL argument");
    LM_CHECK(s->tof.n_bins == 0 || tof != nullptr, LM_ERR_INVALID_ARG, "TOF bins NULL for a TOF scanner");
    LM_CHECK(n >= 1 && n <= s->cfg.max_events, LM_ERR_NOMEM, "frame of %lld events exceeds max_events %lld",
             (long long)n, (long long)s->cfg.max_events);
    LM_CHECK(x0_value > 0.0f, LM_ERR_DOMAIN, "x0_value must be > 0");
    const int count = 2 * s->cfg.n_subsets;
    for (int64_t i = 0; i < (int64_t)s->cfg.epochs * count; ++i)
        LM_CHECK(seqs_host[i] <= s->cfg.n_subsets, LM_ERR_INVALID_ARG, "selection out of range");
    Frame* f = new Frame();
    f->n = n;
    f->x0 = x0_value;
    f->det1.assign(det1, det1 + n);
    f->det2.assign(det2, det2 + n);
    if (tof) f->tof.assign(tof, tof + n);
    else f->tof.assign(n, 0);
    f->corr.assign(n, 1.0f);
    if (corr) std::memcpy(f->corr.data(), corr, n * 4);
    f->contam.assign(contam, contam + n);
    f->seqs.assign(seqs_host, seqs_host + (size_t)s->cfg.epochs * count);
    f->bytes = frame_bytes(s, n);
    f->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        f->ticket = s->next_ticket++;
        s->frames[f->ticket] = f;
        s->queue.push_back(f);
    }
    s->cv_work.notify_all();
    *ticket = f->ticket;
    return LM_OK;
}

int lm_server_wait(lm_server* s, int64_t ticket, float* x_host, double* objective, double* latency_ms,
                   int32_t timeout_ms)
{
    clear_error();
    LM_CHECK(s != nullptr, LM_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->frames.find(ticket);
    LM_CHECK(it != s->frames.end(), LM_ERR_INVALID_ARG, "unknown ticket %lld", (long long)ticket);
    Frame* f = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [&] { return f->done; })) {
        set_error("ticket %lld not finished within %d ms", (long long)ticket, timeout_ms);
        return LM_ERR_TIMEOUT;
    }
    const int status = f->status;
    if (status == LM_OK) {
        if (x_host) std::memcpy(x_host, f->x.data(), f->x.size() * 4);
        if (objective) *objective = f->objective;
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(f->t_done - f->t_submit).count();
    } else {
        set_error("ticket %lld failed: %s", (long long)ticket, f->error.c_str());
    }
    s->frames.erase(it);
    delete f;
    return status;
}

int lm_server_stats(lm_server* s, int64_t* completed, int64_t* in_flight, int64_t* queued, size_t* pool_used,
                    int64_t* max_in_flight)
{
    clear_error();
    LM_CHECK(s != nullptr, LM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (in_flight) *in_flight = (int64_t)s->active.size();
    if (queued) *queued = (int64_t)s->queue.size();
    if (pool_used) *pool_used = s->alloc->used();
    if (max_in_flight) *max_in_flight = s->max_in_flight;
    return LM_OK;
}

int lm_server_destroy(lm_server* s)
{
    clear_error();
    if (!s) return LM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (Frame* f : s->active) {
        if (f->st) {
            lmspdhg_batch_set(s->batch, f->slot, nullptr, s->stream);
            lmspdhg_destroy(f->st);
        }
    }
    for (auto& kv : s->frames) delete kv.second;
    lmspdhg_batch_destroy(s->batch);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->astream);
    delete s->alloc;
    delete s;
    return LM_OK;
}

}  // extern "C"
