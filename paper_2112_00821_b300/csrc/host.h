// Host-side internals of the library shared by the C-ABI layer
// (fassmvs_api.cu) and the serving runtime (server.cu): the context, error
// reporting, scratch management and the batched level loop.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fassmvs.h"
#include "fm_internal.cuh"

struct fassmvs_ctx {
    fassmvs_config cfg;
    int device = 0;
    size_t budget = 0, used = 0;
    std::string err;
    int V = 0;
    double K[9];
    std::vector<double> R, t;
    std::vector<int8_t> side;
    bool cams = false;
    struct Buf { void* p = nullptr; size_t n = 0; };
    std::map<std::string, Buf> bufs;
    cudaStream_t last = nullptr;
    // stage timers
    bool prof = false;
    int inject = 0;                      // test hook (fassmvs_debug_inject)
    int dbg_level = -1;                  // level captured by the next estimate (fassmvs_debug_capture)
    int dbg_dims[5] = {0, 0, 0, 0, 0};  // W, H, D, Ds, G of the captured level
    int dbg_warp_g = -1, dbg_warp_k = -1;   // (plane, view) whose warped values the capture keeps
    struct Rec { cudaEvent_t a, b; int stage; };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    double ms[FASSMVS_NSTAGES] = {};
    uint64_t cnt[FASSMVS_NSTAGES] = {};
    // batched form: work decomposition, graphs, pinned staging of the per-call
    // argument blocks (two halves, each released by an event)
    fassmvs_tuning tune{0, 2, 0};              // automatic chunks and parts
    std::map<uint64_t, fassmvs_tuning> tuned;
    bool graph = false;
    std::map<uint64_t, cudaGraphExec_t> execs;
    std::map<uint64_t, int> seen;
    unsigned char* host_arena[2] = {nullptr, nullptr};
    size_t host_cap = 0;
    cudaEvent_t arena_ev[2] = {nullptr, nullptr};
    int arena_half = 0;
    // host-buffer estimates: two device slots of images and maps, a copy
    // stream each way, and per slot the events "images copied", "estimate
    // done" and "maps copied"
    cudaStream_t hp_h2d = nullptr, hp_d2h = nullptr;
    cudaEvent_t hp_in[2] = {nullptr, nullptr}, hp_comp[2] = {nullptr, nullptr}, hp_out[2] = {nullptr, nullptr};
    int hp_slot = 0;
    size_t hp_slot_bytes = 0;
    // per-frame scratch from the caller (the serving form) instead of by name
    fassmvs_status (*scratch_fn)(void* user, int frame, const char* name, size_t bytes, void** out) = nullptr;
    void* scratch_user = nullptr;
};


namespace fmh {

extern thread_local std::string t_err;

fassmvs_status fail(fassmvs_ctx* c, fassmvs_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
fassmvs_status cuda_check(fassmvs_ctx* c, cudaError_t e, const char* what);
fassmvs_status set_device(fassmvs_ctx* c);
fassmvs_status check_frame(fassmvs_ctx* c, const fassmvs_frame& f, int levels, int idx);

// bump allocator over the two mirrored staging blocks (pinned host, device)
struct Stage {
    unsigned char* host;
    unsigned char* dev;
    size_t off, cap;
    int half;
    void* take(size_t bytes, size_t& at)
    {
        at = (off + 255) & ~(size_t)255;
        off = at + bytes;
        return off <= cap ? host + at : nullptr;
    }
};
fassmvs_status stage_prepare(fassmvs_ctx* c, const fassmvs_frame* frames, int n, int chunk_planes, Stage* out);
// grows both pinned staging halves to at least `bytes` now
fassmvs_status stage_reserve(fassmvs_ctx* c, size_t bytes);
// stage_reserve plus the device mirrors of `bytes` and the work counter
fassmvs_status ctx_reserve(fassmvs_ctx* c, size_t bytes);

// sgm_parts value of the two-pass wavefront aggregation
constexpr int kSgmTwoPass = -1;
// partial sums of the per-direction aggregation for a tuning
int sgm_parts(const fassmvs_tuning& t, int paths);
// what the aggregation of a batch runs as on `device`: 0 for the two-pass
// wavefront form with the winner-takes-all fused (sgm_parts -1, where the
// device launches cooperative kernels), else the partial sums of the
// per-direction form
int agg_parts(const fassmvs_tuning& t, int paths, int device);

// The coarse-to-fine estimate of n frames sharing launches (Sec. 2.1 per
// frame); pyrs, when not NULL, gives resident image pyramids per frame.
fassmvs_status run_batch(fassmvs_ctx* c, const fassmvs_frame* frames, int n, cudaStream_t st,
                         const fassmvs_tuning& tn, const Stage& stage, const fm::PyrSet* pyrs);

// Alg. 3 smoothing weights (a 7-tap Gaussian quantised to a unit sum of 256)
fm::DogWeights dog_weights();

// Largest size over the levels of every per-frame scratch buffer run_batch
// asks for (by name) when the pyramids are resident; parts as agg_parts
// gives, wave_cap = fm::wave_capacity of the device.
void frame_scratch_layout(const fassmvs_config& cfg, int W, int H, int V, int G0, int parts, int wave_cap,
                          std::vector<std::pair<std::string, size_t>>& out);

}  // namespace fmh
