// Serving form of the hot path: frames of a video stream stay resident on the
// device with their image pyramids (built once, on arrival), keyframe
// requests are admitted when their scratch fits the device budget, and
// admitted requests are batched continuously onto several lanes (one stream
// and one context each), so that a batch launched while others run overlaps
// with them on the device.  Each request runs the same coarse-to-fine
// estimate (Sec. 2.1) as fassmvs_estimate, with the same kernels.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.h"
#include "host.h"

namespace {

using namespace fmh;

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SFrame {
    int64_t id;
    int W, H, L;
    double K[9], R[9], t[3];
    size_t off;
    uint8_t* lvl[8];
    int pitch[8];
    cudaEvent_t ready = nullptr;
    int refs = 0;          // requests that name the frame and have not completed
    bool released = false; // the producer will name it no more
};

struct SReq {
    fassmvs_request r;
    std::vector<int64_t> nb;
    std::vector<SFrame*> frames;   // reference first
    std::vector<double> R, t;      // reference -> neighbour
    std::vector<int8_t> side;
    std::vector<std::pair<std::string, size_t>> layout;   // name -> offset in the block
    std::map<std::string, size_t> size_of;
    size_t bytes = 0, off = SIZE_MAX;
    float *d_depth = nullptr, *d_normal = nullptr, *d_conf = nullptr;
    int64_t t_submit = 0, t_admit = 0, t_launch = 0, deadline = 0;
    // post-filters: the kept-depth block (its own arena block, handed to the
    // server's kept maps when the request succeeds), the consistency partners
    // and the relative poses reference -> partner
    size_t keep_bytes = 0, keep_off = SIZE_MAX;
    std::vector<int64_t> geo;
    std::vector<size_t> geo_off;               // arena offsets of the partners' maps (fixed while named)
    std::vector<double> geo_R, geo_t;
};

// a depth map kept for later consistency checks (FASSMVS_POST_KEEP)
struct Kept {
    size_t off = SIZE_MAX;
    int W = 0, H = 0;
    double K[9], R[9], t[3];   // intrinsics and world -> camera pose of its reference
    int refs = 0;              // queued or running requests that name it
    bool released = false;
};

struct Lane {
    fassmvs_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;                 // stream of the current batch
    cudaStream_t prio[4] = {};                 // one stream per priority level, highest first
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<SReq*> batch;
    int64_t t_launch = 0;
    int* h_err = nullptr;                      // pinned: per batch entry, the DoG filter's error word
};

}  // namespace

struct fassmvs_server {
    fassmvs_config cfg;
    fassmvs_server_config scfg;
    int device = 0;
    void* dev_base = nullptr;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::unordered_map<int64_t, std::unique_ptr<SFrame>> frames;
    std::deque<SReq*> pending;    // submitted, waiting for memory
    std::deque<SReq*> admitted;   // scratch reserved, waiting for a lane
    std::deque<fassmvs_result> results;
    std::unordered_map<int64_t, Kept> kept;
    std::vector<Lane> lanes;
    // uploads: host rows -> pinned slot (CPU copy) -> device on copy_st, then
    // the pyramid on pyr_st (highest priority); copies never queue behind
    // kernels, so pushing a frame does not wait for running batches
    cudaStream_t copy_st = nullptr, pyr_st = nullptr;
    struct Slot { unsigned char* host = nullptr; size_t cap = 0; cudaEvent_t done = nullptr; };
    Slot slots[4];
    int next_slot = 0;
    std::mutex up_mu;
    std::thread worker;
    bool stop = false;
    std::string err;
    fassmvs_server_stats stats{};
};

namespace {

fassmvs_status sfail(fassmvs_server* s, fassmvs_status st, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
fassmvs_status sfail(fassmvs_server* s, fassmvs_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    fmh::t_err = buf;
    return st;
}

// scratch of frame f of the lane's current batch: the request's block
fassmvs_status lane_scratch(void* user, int f, const char* name, size_t bytes, void** out)
{
    auto* pr = static_cast<std::pair<fassmvs_server*, Lane*>*>(user);
    fassmvs_server* s = pr->first;
    Lane* ln = pr->second;
    if (f < 0 || f >= (int)ln->batch.size()) return sfail(s, FASSMVS_EINTERNAL, "scratch for frame %d", f);
    SReq* q = ln->batch[f];
    for (auto& kv : q->layout)
        if (kv.first == name) {
            if (bytes > q->size_of[name])
                return sfail(s, FASSMVS_EINTERNAL, "scratch '%s' of %zu bytes exceeds its layout", name, bytes);
            *out = s->arena.at(q->off + kv.second);
            return FASSMVS_OK;
        }
    return sfail(s, FASSMVS_EINTERNAL, "scratch '%s' missing from the layout", name);
}

void mat3_mul(const double* A, const double* B, double* C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0;
            for (int m = 0; m < 3; ++m) v += A[3 * i + m] * B[3 * m + j];
            C[3 * i + j] = v;
        }
}

// completes a request (lock held); frees its block and frame references
void complete(fassmvs_server* s, SReq* q, fassmvs_status st, int batch_size)
{
    fassmvs_result r;
    r.id = q->r.id;
    r.status = st;
    r.batch_size = batch_size;
    r.t_submit_ns = q->t_submit;
    r.t_admit_ns = q->t_admit;
    r.t_launch_ns = q->t_launch;
    r.t_done_ns = now_ns();
    s->results.push_back(r);
    if (q->off != SIZE_MAX) s->arena.release(q->off);
    if (q->keep_off != SIZE_MAX) {
        // (a second request with the same id in flight keeps nothing: the
        // first map stays, the block is given back)
        if (st == FASSMVS_OK && !s->kept.count(q->r.id)) {
            Kept& k = s->kept[q->r.id];
            const SFrame* F0 = q->frames[0];
            k.off = q->keep_off;
            k.W = F0->W;
            k.H = F0->H;
            memcpy(k.K, F0->K, sizeof k.K);
            memcpy(k.R, F0->R, sizeof k.R);
            memcpy(k.t, F0->t, sizeof k.t);
        } else {
            s->arena.release(q->keep_off);
        }
    }
    for (int64_t id : q->geo) {
        auto it = s->kept.find(id);
        if (it == s->kept.end()) continue;
        if (--it->second.refs == 0 && it->second.released) {
            s->arena.release(it->second.off);
            s->kept.erase(it);
        }
    }
    for (SFrame* F : q->frames) {
        if (--F->refs == 0 && F->released) {
            s->arena.release(F->off);
            cudaEventDestroy(F->ready);
            s->frames.erase(F->id);
        }
    }
    if (st == FASSMVS_OK) ++s->stats.completed; else ++s->stats.failed;
    delete q;
}

// launches one batch on a lane (called by the worker without the lock; the
// requests of the batch are owned by the lane meanwhile)
fassmvs_status launch_batch(fassmvs_server* s, Lane& ln, const fassmvs_tuning& tn)
{
    const int n = (int)ln.batch.size();
    std::vector<fassmvs_frame> fr(n);
    std::vector<fm::PyrSet> py(n);
    std::vector<std::vector<const uint8_t*>> nb(n);
    for (int i = 0; i < n; ++i) {
        SReq* q = ln.batch[i];
        SFrame* F0 = q->frames[0];
        const int V = (int)q->nb.size();
        nb[i].resize(V);
        for (int k = 0; k < V; ++k) nb[i][k] = q->frames[k + 1]->lvl[0];
        for (SFrame* F : q->frames)
            if (cudaStreamWaitEvent(ln.st, F->ready, 0) != cudaSuccess)
                return sfail(s, FASSMVS_ECUDA, "wait for frame %lld", (long long)F->id);
        fassmvs_frame& f = fr[i];
        f.ref = F0->lvl[0];
        f.nbrs = nb[i].data();
        f.W = F0->W; f.H = F0->H; f.pitch = F0->pitch[0]; f.n_nb = V;
        f.K = F0->K; f.R = q->R.data(); f.t = q->t.data(); f.side = q->side.data();
        f.planes = q->r.planes;
        f.depth = q->d_depth; f.normal = q->d_normal; f.conf = q->d_conf;
        for (int l = 0; l < F0->L; ++l) {
            py[i].pitch[l] = F0->pitch[l];
            py[i].img[l][0] = F0->lvl[l];
            for (int k = 0; k < V; ++k) py[i].img[l][k + 1] = q->frames[k + 1]->lvl[l];
        }
        if (check_frame(ln.ctx, f, s->cfg.levels, i) != FASSMVS_OK)
            return sfail(s, FASSMVS_EINVAL, "%s", ln.ctx->err.c_str());
    }
    std::pair<fassmvs_server*, Lane*> user{s, &ln};
    ln.ctx->scratch_fn = lane_scratch;
    ln.ctx->scratch_user = &user;
    Stage sg;
    fassmvs_status st = stage_prepare(ln.ctx, fr.data(), n, tn.chunk_planes, &sg);
    if (st == FASSMVS_OK) st = run_batch(ln.ctx, fr.data(), n, ln.st, tn, sg, py.data());
    ln.ctx->scratch_fn = nullptr;
    ln.ctx->scratch_user = nullptr;
    if (st != FASSMVS_OK) return sfail(s, st, "%s", ln.ctx->err.c_str());
    // post-filters (Sec. 2.6) on the outputs, before they are returned
    for (int i = 0; i < n; ++i) {
        SReq* q = ln.batch[i];
        const int pf = q->r.postfilter;
        ln.h_err[i] = 0;
        if (!pf) continue;
        const SFrame* F0 = q->frames[0];
        const int W = F0->W, H = F0->H;
        const size_t np = (size_t)W * H;
        if (pf & FASSMVS_POST_KEEP)
            cudaMemcpyAsync(s->arena.at(q->keep_off), q->d_depth, 4 * np, cudaMemcpyDeviceToDevice, ln.st);
        if (pf & FASSMVS_POST_DOG) {
            auto at = [&](const char* name) -> void* {
                for (auto& kv : q->layout)
                    if (kv.first == name) return s->arena.at(q->off + kv.second);
                return nullptr;
            };
            int* err = (int*)at("dog:err");
            cudaMemsetAsync(err, 0, sizeof(int), ln.st);
            fm::launch_dog_mask(F0->lvl[0], W, H, F0->pitch[0], dog_weights(), (uint8_t*)at("dog:mask"),
                                (uint8_t*)at("dog:tmp"), (int*)at("dog:parent"), (int*)at("dog:size"), err, ln.st);
            fm::launch_apply_mask((const uint8_t*)at("dog:mask"), W, H, q->d_depth, q->d_normal, q->d_conf, ln.st);
            cudaMemcpyAsync(&ln.h_err[i], err, sizeof(int), cudaMemcpyDeviceToHost, ln.st);
        }
        if (pf & FASSMVS_POST_GEO) {
            fm::GeoArgs g;
            memset(&g, 0, sizeof g);
            g.W = W; g.H = H; g.n = (int)q->geo.size(); g.eta_h = q->r.geo_eta_h; g.eta_r = q->r.geo_eta_r;
            g.fx = F0->K[0]; g.fy = F0->K[4]; g.cx = F0->K[2]; g.cy = F0->K[5];
            for (int k = 0; k < g.n; ++k) {
                g.dk[k] = (const float*)s->arena.at(q->geo_off[k]);
                for (int j = 0; j < 9; ++j) g.R[k][j] = q->geo_R[9 * k + j];
                for (int j = 0; j < 3; ++j) g.t[k][j] = q->geo_t[3 * k + j];
            }
            fm::launch_geo_filter(g, q->d_depth, q->d_normal, q->d_conf, nullptr, ln.st);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return sfail(s, FASSMVS_ECUDA, "post-filter launch");
    for (int i = 0; i < n; ++i) {
        SReq* q = ln.batch[i];
        if (!q->r.host_outputs) continue;
        const size_t np = (size_t)q->frames[0]->W * q->frames[0]->H;
        cudaMemcpyAsync(q->r.depth, q->d_depth, 4 * np, cudaMemcpyDeviceToHost, ln.st);
        cudaMemcpyAsync(q->r.normal, q->d_normal, 12 * np, cudaMemcpyDeviceToHost, ln.st);
        cudaMemcpyAsync(q->r.conf, q->d_conf, 4 * np, cudaMemcpyDeviceToHost, ln.st);
    }
    if (cudaEventRecord(ln.done, ln.st) != cudaSuccess) return sfail(s, FASSMVS_ECUDA, "record completion");
    return FASSMVS_OK;
}

void worker(fassmvs_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // retire finished batches
        for (Lane& ln : s->lanes) {
            if (!ln.busy) continue;
            cudaError_t q = cudaEventQuery(ln.done);
            if (q == cudaErrorNotReady) continue;
            const fassmvs_status st = q == cudaSuccess ? FASSMVS_OK : FASSMVS_ECUDA;
            if (st != FASSMVS_OK) s->err = std::string("batch: ") + cudaGetErrorString(q);
            for (size_t i = 0; i < ln.batch.size(); ++i) {
                SReq* r = ln.batch[i];
                // a union-find walk of the DoG filter that reached its bound
                const bool dog_err = st == FASSMVS_OK && (r->r.postfilter & FASSMVS_POST_DOG) && ln.h_err[i];
                if (dog_err) s->err = "request " + std::to_string((long long)r->r.id) + ": DoG filter walk bound";
                complete(s, r, dog_err ? FASSMVS_EINTERNAL : st, (int)ln.batch.size());
            }
            ln.batch.clear();
            ln.busy = false;
            s->cv_done.notify_all();
        }
        // admission in arrival order: a request is admitted once its scratch
        // fits; one that has waited past its deadline fails with ETIMEOUT
        const int64_t t = now_ns();
        while (!s->pending.empty()) {
            SReq* q = s->pending.front();
            if (q->deadline && t > q->deadline) {
                s->pending.pop_front();
                complete(s, q, FASSMVS_ETIMEOUT, 0);
                s->cv_done.notify_all();
                continue;
            }
            size_t off = s->arena.alloc(q->bytes);
            size_t koff = SIZE_MAX;
            if (off != SIZE_MAX && q->keep_bytes) {
                // the kept map outlives the request: from the top, like frames
                koff = s->arena.alloc(q->keep_bytes, true);
                if (koff == SIZE_MAX) {
                    s->arena.release(off);
                    off = SIZE_MAX;
                }
            }
            if (off == SIZE_MAX) {
                // with nothing admitted or running, no completion can free
                // memory for it (the resident frames it needs stay): refuse it
                // rather than wait forever
                bool idle = s->admitted.empty();
                for (Lane& ln : s->lanes) idle = idle && !ln.busy;
                if (!idle) break;
                s->err = "request " + std::to_string((long long)q->r.id) +
                         ": its scratch does not fit next to the resident frames";
                s->pending.pop_front();
                complete(s, q, FASSMVS_ENOMEM, 0);
                s->cv_done.notify_all();
                continue;
            }
            q->off = off;
            q->keep_off = koff;
            q->t_admit = t;
            if (q->r.host_outputs) {
                for (auto& kv : q->layout) {
                    if (kv.first == "out:depth") q->d_depth = (float*)s->arena.at(off + kv.second);
                    if (kv.first == "out:normal") q->d_normal = (float*)s->arena.at(off + kv.second);
                    if (kv.first == "out:conf") q->d_conf = (float*)s->arena.at(off + kv.second);
                }
            }
            s->pending.pop_front();
            s->admitted.push_back(q);
        }
        // continuous batching: every idle lane takes up to max_batch admitted
        // requests now, while the other lanes' batches are still running
        for (Lane& ln : s->lanes) {
            if (ln.busy || s->admitted.empty()) continue;
            int running = 0;
            for (Lane& o : s->lanes) running += o.busy;
            // next to running batches only under a backlog: a lone request
            // waits for the device rather than slowing the running batch down
            if (running > 0 && (int)s->admitted.size() < s->scfg.overlap_queue) break;
            const int m = std::min<int>(s->scfg.max_batch, (int)s->admitted.size());
            for (int i = 0; i < m; ++i) {
                ln.batch.push_back(s->admitted.front());
                s->admitted.pop_front();
            }
            int others = 0;
            for (Lane& o : s->lanes) others += o.busy;
            ln.st = ln.prio[std::min(others, 3)];
            ln.busy = true;
            ln.t_launch = now_ns();
            for (SReq* r : ln.batch) r->t_launch = ln.t_launch;
            ++s->stats.batches;
            s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, m);
            // alone: the fastest decomposition; next to running batches: the
            // one whose short-lived CTAs let the older batch keep priority
            const fassmvs_tuning tn = others ? s->scfg.tuning_overlap : s->scfg.tuning;
            if (others) ++s->stats.overlapped;
            lk.unlock();
            fassmvs_status st = launch_batch(s, ln, tn);
            if (st != FASSMVS_OK) cudaStreamSynchronize(ln.st);   // nothing of it stays in flight
            lk.lock();
            if (st != FASSMVS_OK) {
                for (SReq* r : ln.batch) complete(s, r, st, m);
                ln.batch.clear();
                ln.busy = false;
                s->cv_done.notify_all();
            }
        }
        int busy = 0;
        for (Lane& ln : s->lanes) busy += ln.busy;
        s->stats.bytes_in_use = (int64_t)s->arena.used();
        s->stats.peak_bytes = (int64_t)s->arena.peak();
        if (s->stop && busy == 0) break;
        if (busy) s->cv.wait_for(lk, std::chrono::microseconds(20));
        else if (!s->stop) s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace

extern "C" {

void fassmvs_server_config_default(fassmvs_server_config* c)
{
    if (!c) return;
    c->lanes = 2;
    c->max_batch = 8;
    c->mem_budget = (size_t)16 << 30;
    c->deadline_ms = 0;
    c->overlap_queue = 2;
    c->tuning = fassmvs_tuning{0, 2, 0};
    c->tuning_overlap = fassmvs_tuning{32, 0, 0};
}

fassmvs_status fassmvs_server_create(const fassmvs_config* cfg, const fassmvs_server_config* scfg, int device,
                                     fassmvs_server** out)
{
    if (!cfg || !scfg || !out) return sfail(nullptr, FASSMVS_EINVAL, "NULL argument");
    *out = nullptr;
    if (scfg->lanes < 1 || scfg->lanes > 4) return sfail(nullptr, FASSMVS_EINVAL, "lanes must be 1..4");
    if (scfg->max_batch < 1 || scfg->max_batch > fm::kSgmBatch)
        return sfail(nullptr, FASSMVS_EINVAL, "max_batch must be 1..%d", fm::kSgmBatch);
    if (scfg->mem_budget < 4096) return sfail(nullptr, FASSMVS_EINVAL, "mem_budget below 4 KiB");
    if (scfg->deadline_ms < 0) return sfail(nullptr, FASSMVS_EINVAL, "deadline_ms must be >= 0");
    if (scfg->overlap_queue < 0) return sfail(nullptr, FASSMVS_EINVAL, "overlap_queue must be >= 0");
    // one scratch layout serves both tunings: the same aggregation form
    if ((scfg->tuning.sgm_parts == kSgmTwoPass) != (scfg->tuning_overlap.sgm_parts == kSgmTwoPass) ||
        sgm_parts(scfg->tuning, cfg->paths) != sgm_parts(scfg->tuning_overlap, cfg->paths))
        return sfail(nullptr, FASSMVS_EINVAL, "tuning and tuning_overlap must give the same sgm_parts");
    auto* s = new fassmvs_server();
    s->cfg = *cfg;
    s->scfg = *scfg;
    s->device = device;
    auto bail = [&](fassmvs_status st) {
        std::string e = fmh::t_err;
        fassmvs_server_destroy(s);
        fmh::t_err = e;
        return st;
    };
    for (int i = 0; i < scfg->lanes; ++i) {
        Lane ln;
        fassmvs_status st = fassmvs_create(cfg, device, 0, &ln.ctx);
        if (st != FASSMVS_OK) return bail(st);
        st = fassmvs_set_tuning(ln.ctx, &scfg->tuning);
        // staging (pinned halves and their device mirrors, 16 MB each: batches of
        // several 4K frames) and the work counter reserved up front, outside the
        // admission budget: growing them later would call cudaFree, which waits
        // for every lane's running batch
        if (st == FASSMVS_OK) st = ctx_reserve(ln.ctx, (size_t)16 << 20);
        if (st == FASSMVS_OK) st = fassmvs_set_tuning(ln.ctx, &scfg->tuning_overlap);   // validates it
        // a batch launched while k others run goes to priority level k, so
        // the oldest batch keeps the SMs and newer ones fill what it leaves
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        for (int k = 0; k < 4 && st == FASSMVS_OK; ++k) {
            const int pr = std::min(least, greatest + k);
            if (cudaStreamCreateWithPriority(&ln.prio[k], cudaStreamNonBlocking, pr) != cudaSuccess)
                st = sfail(s, FASSMVS_ECUDA, "stream");
        }
        ln.st = ln.prio[0];
        if (st == FASSMVS_OK && cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess)
            st = sfail(s, FASSMVS_ECUDA, "event");
        if (st == FASSMVS_OK &&
            cudaHostAlloc((void**)&ln.h_err, sizeof(int) * fm::kSgmBatch, cudaHostAllocDefault) != cudaSuccess)
            st = sfail(s, FASSMVS_ECUDA, "pinned error words");
        s->lanes.push_back(ln);
        if (st != FASSMVS_OK) return bail(st);
    }
    {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s->pyr_st, cudaStreamNonBlocking, greatest) != cudaSuccess)
            return bail(sfail(s, FASSMVS_ECUDA, "stream"));
        for (auto& sl : s->slots)
            if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
                return bail(sfail(s, FASSMVS_ECUDA, "event"));
    }
    if (cudaMalloc(&s->dev_base, scfg->mem_budget) != cudaSuccess) {
        cudaGetLastError();
        s->dev_base = nullptr;
        return bail(sfail(s, FASSMVS_ENOMEM, "cannot reserve %zu device bytes", scfg->mem_budget));
    }
    s->arena.init(scfg->mem_budget, s->dev_base);
    s->stats.capacity = (int64_t)scfg->mem_budget;
    s->worker = std::thread(worker, s);
    *out = s;
    return FASSMVS_OK;
}

void fassmvs_server_destroy(fassmvs_server* s)
{
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stop = true;
        }
        s->cv.notify_all();
        s->worker.join();
    }
    for (SReq* q : s->pending) delete q;
    for (SReq* q : s->admitted) delete q;
    for (Lane& ln : s->lanes) {
        for (cudaStream_t q : ln.prio)
            if (q) cudaStreamSynchronize(q);
        if (ln.ctx) fassmvs_destroy(ln.ctx);
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.h_err) cudaFreeHost(ln.h_err);
        for (cudaStream_t q : ln.prio)
            if (q) cudaStreamDestroy(q);
    }
    for (cudaStream_t q : {s->copy_st, s->pyr_st})
        if (q) {
            cudaStreamSynchronize(q);
            cudaStreamDestroy(q);
        }
    for (auto& sl : s->slots) {
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (auto& kv : s->frames)
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
    if (s->dev_base) cudaFree(s->dev_base);
    delete s;
}

fassmvs_status fassmvs_server_push_frame(fassmvs_server* s, int64_t id, const uint8_t* img, int W, int H,
                                         int pitch, const double K[9], const double R[9], const double t[3])
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    if (!img || !K || !R || !t) return sfail(s, FASSMVS_EINVAL, "NULL argument");
    const int L = s->cfg.levels;
    if (W < 2 || H < 2 || W > 8192 || H > 8192 || pitch < W) return sfail(s, FASSMVS_EINVAL, "bad frame size");
    if (((W - 1) >> (L - 1)) + 1 < 2 || ((H - 1) >> (L - 1)) + 1 < 2)
        return sfail(s, FASSMVS_EINVAL, "frame too small for %d levels", L);
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(R[i]) || !std::isfinite(K[i])) return sfail(s, FASSMVS_EINVAL, "pose is not finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(t[i])) return sfail(s, FASSMVS_EINVAL, "pose is not finite");
    auto F = std::make_unique<SFrame>();
    F->id = id; F->W = W; F->H = H; F->L = L;
    memcpy(F->K, K, sizeof F->K);
    memcpy(F->R, R, sizeof F->R);
    memcpy(F->t, t, sizeof F->t);
    size_t offs[8], total = 0;
    int w = W, h = H;
    for (int l = 0; l < L; ++l) {
        if (l > 0) { w = (w + 1) / 2; h = (h + 1) / 2; }
        offs[l] = total;
        // levels >= 1 in 16-byte rows (the cost kernel stages them by TMA);
        // level 0 keeps the pushed frame's layout
        F->pitch[l] = l ? (w + 15) & ~15 : w;
        total += align_up((size_t)F->pitch[l] * h);
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->frames.count(id)) return sfail(s, FASSMVS_EINVAL, "frame %lld pushed twice", (long long)id);
        F->off = s->arena.alloc(total, true);
        if (F->off == SIZE_MAX)
            return sfail(s, FASSMVS_EBUSY, "no room for frame %lld (%zu of %zu bytes in use)", (long long)id,
                         s->arena.used(), s->arena.capacity());
    }
    for (int l = 0; l < L; ++l) F->lvl[l] = s->arena.at(F->off + offs[l]);
    cudaSetDevice(s->device);
    cudaError_t e = cudaSuccess;
    {
        std::lock_guard<std::mutex> ug(s->up_mu);
        auto& sl = s->slots[s->next_slot];
        s->next_slot = (s->next_slot + 1) % 4;
        e = cudaEventSynchronize(sl.done);               // its previous copy has left the slot
        const size_t need = (size_t)W * H;
        if (e == cudaSuccess && sl.cap < need) {
            if (sl.host) cudaFreeHost(sl.host);
            sl.host = nullptr;
            sl.cap = 0;
            e = cudaHostAlloc((void**)&sl.host, need, cudaHostAllocDefault);
            if (e == cudaSuccess) sl.cap = need;
        }
        if (e == cudaSuccess) {
            for (int y = 0; y < H; ++y) memcpy(sl.host + (size_t)y * W, img + (size_t)y * pitch, W);
            e = cudaMemcpyAsync(F->lvl[0], sl.host, need, cudaMemcpyHostToDevice, s->copy_st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(sl.done, s->copy_st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->pyr_st, sl.done, 0);
    }
    int ws = W, hs = H;
    for (int l = 1; l < L && e == cudaSuccess; ++l) {
        fm::launch_pyramid_down(F->lvl[l - 1], ws, hs, F->pitch[l - 1], F->lvl[l], F->pitch[l], s->pyr_st);
        ws = (ws + 1) / 2;
        hs = (hs + 1) / 2;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&F->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(F->ready, s->pyr_st);
    std::lock_guard<std::mutex> g(s->mu);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s->copy_st);
        cudaStreamSynchronize(s->pyr_st);
        s->arena.release(F->off);
        if (F->ready) cudaEventDestroy(F->ready);
        return sfail(s, FASSMVS_ECUDA, "frame upload: %s", cudaGetErrorString(e));
    }
    s->frames[id] = std::move(F);
    ++s->stats.frames;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_server_release_frame(fassmvs_server* s, int64_t id)
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->frames.find(id);
    if (it == s->frames.end() || it->second->released)
        return sfail(s, FASSMVS_EINVAL, "frame %lld is not resident", (long long)id);
    SFrame* F = it->second.get();
    F->released = true;
    if (F->refs == 0) {
        // no request names it: wait for its own upload before reusing the memory
        cudaEventSynchronize(F->ready);
        s->arena.release(F->off);
        cudaEventDestroy(F->ready);
        s->frames.erase(it);
    }
    return FASSMVS_OK;
}

fassmvs_status fassmvs_server_submit(fassmvs_server* s, const fassmvs_request* r)
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    if (!r) return sfail(s, FASSMVS_EINVAL, "request is NULL");
    if (r->n_nb < 1 || r->n_nb > fm::kMaxViews || !r->nbrs)
        return sfail(s, FASSMVS_EINVAL, "request %lld: 1..%d neighbour frames", (long long)r->id, fm::kMaxViews);
    if (!r->depth || !r->normal || !r->conf) return sfail(s, FASSMVS_EINVAL, "request %lld: NULL output", (long long)r->id);
    // outputs: pinned host memory (copied back asynchronously) or device memory
    for (const void* p : {(const void*)r->depth, (const void*)r->normal, (const void*)r->conf}) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); at.type = cudaMemoryTypeUnregistered; }
        const bool ok = r->host_outputs ? at.type == cudaMemoryTypeHost : at.type == cudaMemoryTypeDevice;
        if (!ok)
            return sfail(s, FASSMVS_EINVAL, "request %lld: outputs must be %s memory", (long long)r->id,
                         r->host_outputs ? "pinned host" : "device");
    }
    const int pf = r->postfilter;
    if (pf & ~(FASSMVS_POST_DOG | FASSMVS_POST_GEO | FASSMVS_POST_KEEP))
        return sfail(s, FASSMVS_EINVAL, "request %lld: unknown post-filter flags", (long long)r->id);
    if ((pf & FASSMVS_POST_GEO) && (r->geo_n < 1 || r->geo_n > 4 || !(r->geo_eta_r > 0.0) || r->geo_eta_h < 0))
        return sfail(s, FASSMVS_EINVAL, "request %lld: geo_n 1..4, geo_eta_r > 0, geo_eta_h >= 0", (long long)r->id);
    auto q = std::make_unique<SReq>();
    q->r = *r;
    q->nb.assign(r->nbrs, r->nbrs + r->n_nb);
    q->r.nbrs = nullptr;
    const fassmvs_planes& pl = r->planes;
    const int L = s->cfg.levels;
    if (pl.G0 < 1 || (pl.G0 - 1) / (1 << (L - 1)) + 1 > fm::kMaxSlots)
        return sfail(s, FASSMVS_EINVAL, "request %lld: G0 out of range", (long long)r->id);
    if (!(std::isfinite(pl.rho_far) && std::isfinite(pl.drho)) ||
        !(pl.rho_far > 0.0 || (pl.rho_far >= 0.0 && pl.drho > 0.0)))
        return sfail(s, FASSMVS_EINVAL, "request %lld: bad plane list", (long long)r->id);
    std::lock_guard<std::mutex> g(s->mu);
    auto find = [&](int64_t id) -> SFrame* {
        auto it = s->frames.find(id);
        return it == s->frames.end() || it->second->released ? nullptr : it->second.get();
    };
    SFrame* F0 = find(r->ref);
    if (!F0) return sfail(s, FASSMVS_EINVAL, "request %lld: frame %lld is not resident", (long long)r->id, (long long)r->ref);
    q->frames.push_back(F0);
    for (int64_t id : q->nb) {
        SFrame* F = find(id);
        if (!F || id == r->ref)
            return sfail(s, FASSMVS_EINVAL, "request %lld: neighbour %lld is not resident", (long long)r->id, (long long)id);
        if (F->W != F0->W || F->H != F0->H || memcmp(F->K, F0->K, sizeof F->K) != 0)
            return sfail(s, FASSMVS_EINVAL, "request %lld: frame %lld differs in size or intrinsics", (long long)r->id,
                         (long long)id);
        q->frames.push_back(F);
    }
    // relative poses: X_k = R_k R_ref^T X_ref + (t_k - R_k R_ref^T t_ref)
    double RrT[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) RrT[3 * i + j] = F0->R[3 * j + i];
    for (size_t k = 0; k < q->nb.size(); ++k) {
        const SFrame* F = q->frames[k + 1];
        double Rk[9];
        mat3_mul(F->R, RrT, Rk);
        for (int i = 0; i < 9; ++i) q->R.push_back(Rk[i]);
        for (int i = 0; i < 3; ++i) {
            double v = F->t[i];
            for (int m = 0; m < 3; ++m) v -= Rk[3 * i + m] * F0->t[m];
            q->t.push_back(v);
        }
        q->side.push_back(q->nb[k] < r->ref ? -1 : 1);
    }
    // consistency partners: kept depth maps of the same size and intrinsics;
    // X_k = R_k R_ref^T X_ref + (t_k - R_k R_ref^T t_ref) as for the views
    if (pf & FASSMVS_POST_GEO) {
        for (int i = 0; i < r->geo_n; ++i) {
            auto it = s->kept.find(r->geo_ids[i]);
            if (it == s->kept.end() || it->second.released)
                return sfail(s, FASSMVS_EINVAL, "request %lld: no depth map of request %lld is kept", (long long)r->id,
                             (long long)r->geo_ids[i]);
            const Kept& k = it->second;
            if (k.W != F0->W || k.H != F0->H || memcmp(k.K, F0->K, sizeof k.K) != 0)
                return sfail(s, FASSMVS_EINVAL, "request %lld: kept map %lld differs in size or intrinsics",
                             (long long)r->id, (long long)r->geo_ids[i]);
            double Rk[9];
            mat3_mul(k.R, RrT, Rk);
            for (int j = 0; j < 9; ++j) q->geo_R.push_back(Rk[j]);
            for (int a = 0; a < 3; ++a) {
                double v = k.t[a];
                for (int m = 0; m < 3; ++m) v -= Rk[3 * a + m] * F0->t[m];
                q->geo_t.push_back(v);
            }
            q->geo.push_back(r->geo_ids[i]);
            q->geo_off.push_back(k.off);
        }
    }
    if ((pf & FASSMVS_POST_KEEP) && s->kept.count(r->id))
        return sfail(s, FASSMVS_EINVAL, "request %lld: a depth map of that id is already kept", (long long)r->id);
    // scratch layout of the request
    std::vector<std::pair<std::string, size_t>> sizes;
    frame_scratch_layout(s->cfg, F0->W, F0->H, (int)q->nb.size(), pl.G0,
                         agg_parts(s->scfg.tuning, s->cfg.paths, s->device), fm::wave_capacity(s->device), sizes);
    if (r->host_outputs) {
        const size_t np = (size_t)F0->W * F0->H;
        sizes.push_back({"out:depth", 4 * np});
        sizes.push_back({"out:normal", 12 * np});
        sizes.push_back({"out:conf", 4 * np});
    } else {
        q->d_depth = r->depth;
        q->d_normal = r->normal;
        q->d_conf = r->conf;
    }
    const size_t np0 = (size_t)F0->W * F0->H;
    if (pf & FASSMVS_POST_DOG) {
        sizes.push_back({"dog:mask", np0});
        sizes.push_back({"dog:tmp", np0});
        sizes.push_back({"dog:parent", 4 * np0});
        sizes.push_back({"dog:size", 4 * np0});
        sizes.push_back({"dog:err", sizeof(int)});
    }
    if (pf & FASSMVS_POST_KEEP) q->keep_bytes = 4 * np0;
    size_t off = 0;
    for (auto& kv : sizes) {
        q->layout.push_back({kv.first, off});
        q->size_of[kv.first] = kv.second;
        off += align_up(kv.second);
    }
    q->bytes = off;
    if (q->bytes + align_up(q->keep_bytes) > s->arena.capacity())
        return sfail(s, FASSMVS_ENOMEM, "request %lld needs %zu bytes, more than the %zu-byte budget", (long long)r->id,
                     q->bytes + align_up(q->keep_bytes), s->arena.capacity());
    for (SFrame* F : q->frames) ++F->refs;
    for (int64_t id : q->geo) ++s->kept[id].refs;
    q->t_submit = now_ns();
    q->deadline = s->scfg.deadline_ms ? q->t_submit + (int64_t)s->scfg.deadline_ms * 1000000 : 0;
    s->pending.push_back(q.release());
    ++s->stats.submitted;
    s->cv.notify_all();
    return FASSMVS_OK;
}

fassmvs_status fassmvs_server_cancel(fassmvs_server* s, int64_t id)
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    for (std::deque<SReq*>* dq : {&s->pending, &s->admitted})
        for (auto it = dq->begin(); it != dq->end(); ++it)
            if ((*it)->r.id == id) {
                SReq* q = *it;
                dq->erase(it);
                complete(s, q, FASSMVS_ECANCELED, 0);
                s->cv.notify_all();        // memory may have come free for the next in line
                s->cv_done.notify_all();
                return FASSMVS_OK;
            }
    for (Lane& ln : s->lanes)
        for (SReq* q : ln.batch)
            if (q->r.id == id) return sfail(s, FASSMVS_EBUSY, "request %lld is running", (long long)id);
    return sfail(s, FASSMVS_EINVAL, "no queued or running request %lld", (long long)id);
}

fassmvs_status fassmvs_server_release_depth(fassmvs_server* s, int64_t id)
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->kept.find(id);
    if (it == s->kept.end() || it->second.released)
        return sfail(s, FASSMVS_EINVAL, "no depth map of request %lld is kept", (long long)id);
    if (it->second.refs == 0) {
        s->arena.release(it->second.off);
        s->kept.erase(it);
        s->cv.notify_all();                    // memory may have come free for the next in line
    } else {
        it->second.released = true;
    }
    return FASSMVS_OK;
}

fassmvs_status fassmvs_server_poll(fassmvs_server* s, fassmvs_result* out, int max, int* n_out, int timeout_ms)
{
    if (!s) return sfail(nullptr, FASSMVS_EINVAL, "server is NULL");
    if (!out || !n_out || max < 1) return sfail(s, FASSMVS_EINVAL, "bad poll arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->results.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !s->results.empty(); });
    int n = 0;
    while (n < max && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    *n_out = n;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_server_get_stats(fassmvs_server* s, fassmvs_server_stats* st)
{
    if (!s || !st) return sfail(s, FASSMVS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    *st = s->stats;
    st->bytes_in_use = (int64_t)s->arena.used();
    st->peak_bytes = (int64_t)s->arena.peak();
    st->queued = (int64_t)(s->pending.size() + s->admitted.size());
    st->resident_frames = (int64_t)s->frames.size();
    return FASSMVS_OK;
}

const char* fassmvs_server_last_error(const fassmvs_server* s)
{
    return s ? s->err.c_str() : fmh::t_err.c_str();
}

}  // extern "C"
