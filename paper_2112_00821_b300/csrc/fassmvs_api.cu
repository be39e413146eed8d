// C-ABI layer of the B300 FaSS-MVS library: argument validation, the host-side
// FP64 camera algebra (rank-1 homography factors), scratch management within
// the context's memory budget, and the coarse-to-fine level loop of Sec. 2.1.
// Every compute step runs in the kernels of cost.cu, sgm.cu and stages.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <vector>
#include <atomic>

#include <cuda.h>   // CUtensorMap and its enums; the encoder is resolved through the runtime
#include <nvtx3/nvToolsExt.h>   // header-only ranges for profilers (no-ops without one)

#include "../../include/fassmvs.h"
#include "fm_internal.cuh"
#include "host.h"

using namespace fmh;

namespace fm {
static std::atomic<uint64_t> g_launches{0};
uint64_t launches() { return g_launches.load(); }
void count_launch(int n) { g_launches.fetch_add((uint64_t)n); }
}  // namespace fm


namespace fmh {

thread_local std::string t_err;

fassmvs_status fail(fassmvs_ctx* c, fassmvs_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    t_err = buf;
    return s;
}

}  // namespace fmh

void fm::set_error(const char* msg) { fmh::t_err = msg; }

namespace fmh {

fassmvs_status cuda_check(fassmvs_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return FASSMVS_OK;
    return fail(c, FASSMVS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FM_TRY(expr)                          \
    do {                                      \
        fassmvs_status _s = (expr);           \
        if (_s != FASSMVS_OK) return _s;      \
    } while (0)

// cuTensorMapEncodeTiled, resolved once through the runtime (no link against
// the driver library); null when the driver does not offer it
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// the tensor map of a uint8 view image for the cost kernel's staging box;
// false when the image cannot be staged (row pitch or base not 16-byte
// aligned, image smaller than the box, or no encoder)
bool encode_view(void* out, const uint8_t* img, int W, int H, int pitch)
{
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || ((uintptr_t)img & 15) || (pitch & 15) || W < fm::kStageBX || H < fm::kStageBY) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)fm::kStageBX, (cuuint32_t)fm::kStageBY};
    const cuuint32_t es[2] = {1, 1};
    return fn(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(img), dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// device scratch kept by name; grows within the budget
fassmvs_status ensure(fassmvs_ctx* c, const char* name, size_t bytes, void** out)
{
    auto& b = c->bufs[name];
    if (b.n >= bytes && b.p) { *out = b.p; return FASSMVS_OK; }
    size_t need = bytes + 256;
    if (c->budget && c->used - b.n + need > c->budget)
        return fail(c, FASSMVS_ENOMEM, "scratch '%s' of %zu bytes exceeds the memory budget (%zu of %zu used)",
                    name, bytes, c->used, c->budget);
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        c->used -= b.n;
        b.p = nullptr;
        b.n = 0;
        FM_TRY(cuda_check(c, e, "cudaFree"));
    }
    void* p = nullptr;
    FM_TRY(cuda_check(c, cudaMalloc(&p, need), "cudaMalloc"));
    b.p = p;
    b.n = need;
    c->used += need;
    *out = p;
    return FASSMVS_OK;
}

cudaEvent_t take_event(fassmvs_ctx* c)
{
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// an NVTX range for a scope (levels of the coarse-to-fine loop)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Brackets the launches of one stage with events when profiling is on, and
// with an NVTX range named after the stage (seen by nsys / ncu when attached).
const char* const kStageNames[8] = {"fassmvs pyramid", "fassmvs census", "fassmvs cost",    "fassmvs sgm",
                                    "fassmvs wta",     "fassmvs median", "fassmvs normals", "fassmvs window"};
struct StageTimer {
    fassmvs_ctx* c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(fassmvs_ctx* c_, int s, cudaStream_t st_) : c(c_), stage(s), st(st_)
    {
        nvtxRangePushA(s >= 0 && s < 8 ? kStageNames[s] : "fassmvs stage");
        if (c && c->prof && (a = take_event(c))) cudaEventRecord(a, st);
    }
    ~StageTimer()
    {
        nvtxRangePop();
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) { c->pool.push_back(a); return; }
        cudaEventRecord(b, st);
        c->pending.push_back({a, b, stage});
    }
};

fassmvs_status set_device(fassmvs_ctx* c) { return cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"); }

// largest cost one view can contribute (census Hamming or NCC)
int cost_max(int cost) { return cost ? 255 : fm::kCensusMax; }

fassmvs_status check_config(fassmvs_ctx* c, const fassmvs_config* cfg)
{
    if (!cfg) return fail(c, FASSMVS_EINVAL, "config is NULL");
    if (cfg->levels < 1 || cfg->levels > 8) return fail(c, FASSMVS_EINVAL, "levels must be 1..8");
    for (int l = 0; l < cfg->levels - 1; ++l)
        if (cfg->D[l] < 1 || cfg->D[l] > fm::kMaxSlots)
            return fail(c, FASSMVS_EINVAL, "D[%d] must be 1..%d", l, fm::kMaxSlots);
    if (cfg->paths != 8 && cfg->paths != 4) return fail(c, FASSMVS_EINVAL, "paths must be 4 or 8");
    if (cfg->variant < 0 || cfg->variant > 2) return fail(c, FASSMVS_EINVAL, "variant must be 0, 1 or 2");
    if (cfg->p1 < 0 || cfg->p2 < 0) return fail(c, FASSMVS_EINVAL, "penalties must be >= 0");
    if (cfg->normal_radius < 0 || cfg->normal_radius > 8) return fail(c, FASSMVS_EINVAL, "normal_radius must be 0..8");
    if (cfg->dmax < 0 || cfg->dmax > 127) return fail(c, FASSMVS_EINVAL, "dmax must be 0..127");
    if (!(cfg->beta > 0) || !(cfg->normal_beta > 0)) return fail(c, FASSMVS_EINVAL, "beta must be > 0");
    if (cfg->cost != 0 && cfg->cost != 1) return fail(c, FASSMVS_EINVAL, "cost must be 0 (census) or 1 (NCC)");
    return FASSMVS_OK;
}

// K^-1 of an upper-triangular intrinsic matrix (zero skew allowed or not)
bool k_inverse(const double K[9], double Ki[9])
{
    if (K[3] != 0.0 || K[6] != 0.0 || K[7] != 0.0 || K[8] != 1.0 || K[0] == 0.0 || K[4] == 0.0) return false;
    const double fx = K[0], s = K[1], cx = K[2], fy = K[4], cy = K[5];
    Ki[0] = 1.0 / fx; Ki[1] = -s / (fx * fy); Ki[2] = (s * cy - cx * fy) / (fx * fy);
    Ki[3] = 0.0;      Ki[4] = 1.0 / fy;       Ki[5] = -cy / fy;
    Ki[6] = 0.0;      Ki[7] = 0.0;            Ki[8] = 1.0;
    return true;
}

// Rank-1 factors of H(rho) = K R K^-1 - rho (K t)(n^T K^-1) per view.
fassmvs_status view_geom(fassmvs_ctx* c, const double K[9], int V, const double* R, const double* t,
                         const double n[3], fm::ViewGeom* vg)
{
    double Ki[9];
    if (!k_inverse(K, Ki)) return fail(c, FASSMVS_EINVAL, "K must be [[fx s cx][0 fy cy][0 0 1]] with fx, fy != 0");
    for (int k = 0; k < V; ++k) {
        const double* Rk = R + 9 * k;
        const double* tk = t + 3 * k;
        double KR[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int m = 0; m < 3; ++m) s += K[3 * i + m] * Rk[3 * m + j];
                KR[3 * i + j] = s;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0;
                for (int m = 0; m < 3; ++m) s += KR[3 * i + m] * Ki[3 * m + j];
                vg->A[k][3 * i + j] = s;
            }
        for (int i = 0; i < 3; ++i) {
            double s = 0;
            for (int m = 0; m < 3; ++m) s += K[3 * i + m] * tk[m];
            vg->e[k][i] = s;
        }
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int m = 0; m < 3; ++m) s += n[m] * Ki[3 * m + j];
            vg->c[k][j] = s;
        }
    }
    return FASSMVS_OK;
}

fm::Intr intr(const double K[9]) { return fm::Intr{(float)K[0], (float)K[4], (float)K[2], (float)K[5]}; }

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

fassmvs_status launch_status(fassmvs_ctx* c, const char* what)
{
    return cuda_check(c, cudaGetLastError(), what);
}

fassmvs_status cost_volume_impl(fassmvs_ctx* c, const uint8_t* ref, const uint8_t* const* nbrs, int V,
                                const int8_t* side, int W, int H, int pitch, const double K[9],
                                const double* R, const double* t, const double n[3], double rho0,
                                double drho, int G, const int32_t* lo, int D, int Ds, uint16_t* Sv,
                                cudaStream_t st)
{
    if (!ref || !nbrs || !side || !K || !R || !t || !n || !Sv) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (W < 2 || H < 2) return fail(c, FASSMVS_EINVAL, "image must be at least 2x2");
    if (W > 8192 || H > 8192) return fail(c, FASSMVS_EINVAL, "images up to 8192 pixels per side");
    if (pitch < W) return fail(c, FASSMVS_EINVAL, "pitch < W");
    if (V < 1 || V > fm::kMaxViews) return fail(c, FASSMVS_EINVAL, "1..%d neighbour views", fm::kMaxViews);
    if (D < 1 || D > fm::kMaxSlots || G < D || Ds < D) return fail(c, FASSMVS_EINVAL, "need 1 <= D <= 256, D <= G, D <= Ds");
    if (!lo && G != D) return fail(c, FASSMVS_EINVAL, "without a window map the level sweeps all G = D planes");
    if (!(std::isfinite(rho0) && std::isfinite(drho)) || !(rho0 > 0.0 || (rho0 >= 0.0 && drho > 0.0)))
        return fail(c, FASSMVS_EINVAL, "plane list must have positive inverse distances");
    for (int k = 0; k < V; ++k)
        if (!nbrs[k]) return fail(c, FASSMVS_EINVAL, "neighbour %d is NULL", k);
    fm::ViewGeom vg;
    FM_TRY(view_geom(c, K, V, R, t, n, &vg));
    fm::LevelPlanes lp{rho0, drho, G, V, 0.5 * (W - 1), 0.5 * (H - 1)};
    void *htab, *delta, *cref;
    FM_TRY(ensure(c, "htab", sizeof(float) * 18 * (size_t)G * V, &htab));
    FM_TRY(ensure(c, "delta", sizeof(float) * (size_t)G, &delta));
    FM_TRY(ensure(c, "cref", sizeof(uint64_t) * (size_t)W * H, &cref));
    {
        StageTimer tm(c, FASSMVS_STAGE_CENSUS, st);
        fm::launch_prep_level(vg, lp, (float*)htab, (float*)delta, st);
        fm::launch_census(ref, W, H, pitch, (uint64_t*)cref, st);
    }
    fm::CostArgs a;
    memset(&a, 0, sizeof a);
    a.cost = c->cfg.cost;
    a.ref = ref;
    a.ref_pitch = pitch;
    a.cref = (const uint64_t*)cref;
    int nL = 0, nR = 0;
    for (int k = 0; k < V; ++k) {
        a.views.img[k] = nbrs[k];
        a.views.side[k] = side[k] < 0 ? -1 : 1;
        if (side[k] < 0) ++nL; else ++nR;
    }
    a.V = V; a.W = W; a.H = H; a.pitch = pitch;
    a.nL = nL; a.nR = nR; a.nmax = nL > nR ? nL : nR;
    a.mL = nL ? ((1ull << 32) + nL - 1) / nL : 0;
    a.mR = nR ? ((1ull << 32) + nR - 1) / nR : 0;
    a.htab = (const float*)htab;
    a.lo = lo;
    a.D = D; a.Ds = Ds; a.G = G;
    a.pstride = (size_t)Ds;
    a.bstride = 8;
    a.bshift = 3;
    a.S = Sv;
    StageTimer tm(c, FASSMVS_STAGE_COST, st);
    fm::launch_cost(a, st);
    return launch_status(c, "cost volume launch");
}

fassmvs_status sgm_impl(fassmvs_ctx* c, const uint16_t* Sv, const int32_t* lo, const int8_t* dI,
                        const uint8_t* img, int img_pitch, int W, int H, int D, int Ds,
                        const fassmvs_sgm_params* prm, int Smax, uint16_t* Sbar, cudaStream_t st)
{
    if (!Sv || !Sbar || !prm) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (W < 1 || H < 1) return fail(c, FASSMVS_EINVAL, "empty image");
    if (D < 1 || D > fm::kMaxSlots || Ds < D || (Ds & 7)) return fail(c, FASSMVS_EINVAL, "need 1 <= D <= 256, Ds >= D, Ds %% 8 == 0");
    if ((reinterpret_cast<uintptr_t>(Sv) | reinterpret_cast<uintptr_t>(Sbar)) & 15)
        return fail(c, FASSMVS_EINVAL, "volumes must be 16-byte aligned");
    if (prm->paths != 8 && prm->paths != 4) return fail(c, FASSMVS_EINVAL, "paths must be 4 or 8");
    if (prm->variant < 0 || prm->variant > 2) return fail(c, FASSMVS_EINVAL, "variant must be 0..2");
    if (prm->variant == 1 && !dI) return fail(c, FASSMVS_EINVAL, "surface-normal variant needs dI");
    if (prm->p2_lut && !img) return fail(c, FASSMVS_EINVAL, "adaptive phi2 needs the level image");
    if (prm->p1 < 0 || prm->p2 < 0 || prm->dmax < 0) return fail(c, FASSMVS_EINVAL, "negative penalty or dmax");
    fm::SgmArgs a;
    memset(&a, 0, sizeof a);
    int p2max = prm->p2;
    if (prm->p2_lut) {
        a.use_lut = 1;
        p2max = 0;
        for (int i = 0; i < 256; ++i) {
            a.lut[i] = prm->p2_lut[i];
            if (a.lut[i] > p2max) p2max = a.lut[i];
        }
    }
    if (p2max < prm->p1) p2max = prm->p1;
    if ((long long)prm->paths * (Smax + p2max) >= 65536)
        return fail(c, FASSMVS_EINVAL, "aggregated costs could exceed 16 bits: paths %d x (%d + %d)", prm->paths, Smax, p2max);
    a.S = Sv; a.lo = lo; a.dI = dI; a.img = img; a.img_pitch = img_pitch;
    a.W = W; a.H = H; a.D = D; a.Ds = Ds;
    a.pstride = (size_t)Ds;
    a.bstride = 8;
    a.bshift = 3;
    a.paths = prm->paths; a.variant = prm->variant; a.p1 = prm->p1; a.p2 = prm->p2; a.dmax = prm->dmax;
    a.Sbar = Sbar;
    StageTimer tm(c, FASSMVS_STAGE_SGM, st);
    fm::launch_sgm(a, st);
    return launch_status(c, "sgm launch");
}

void p2_table(int p1, double alpha, double beta, uint16_t* lut)
{
    for (int d = 0; d < 256; ++d) {
        double v = std::floor((double)p1 * (1.0 + alpha * std::exp(-(double)d / beta)) + 0.5);
        lut[d] = (uint16_t)(v > 65535.0 ? 65535.0 : v);
    }
}

}  // namespace fmh

// ===================================================================== ABI
extern "C" {

fassmvs_status fassmvs_config_default(fassmvs_config* cfg)
{
    if (!cfg) return fail(nullptr, FASSMVS_EINVAL, "config is NULL");
    memset(cfg, 0, sizeof *cfg);
    cfg->levels = 1;
    for (int i = 0; i < 8; ++i) cfg->D[i] = 256;
    cfg->paths = 8;
    cfg->variant = 0;
    cfg->p1 = 24;
    cfg->p2 = 0;
    cfg->adaptive_p2 = 1;
    cfg->alpha = 8.0f;
    cfg->beta = 10.0f;
    cfg->median5 = 1;
    cfg->normal_radius = 2;
    cfg->normal_beta = 10.0f;
    cfg->rho_deg = 60.0f;
    cfg->dmax = 8;
    cfg->cost = 0;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_create(const fassmvs_config* cfg, int device, size_t mem_budget, fassmvs_ctx** out)
{
    if (!out) return fail(nullptr, FASSMVS_EINVAL, "out is NULL");
    *out = nullptr;
    fassmvs_ctx* c = new (std::nothrow) fassmvs_ctx();
    if (!c) return fail(nullptr, FASSMVS_ENOMEM, "host allocation failed");
    fassmvs_config def;
    fassmvs_config_default(&def);
    fassmvs_status s = check_config(c, cfg ? cfg : &def);
    if (s != FASSMVS_OK) { delete c; return s; }
    c->cfg = cfg ? *cfg : def;
    c->device = device;
    c->budget = mem_budget;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        delete c;
        return fail(nullptr, FASSMVS_ECUDA, "no CUDA device %d", device);
    }
    s = set_device(c);
    if (s != FASSMVS_OK) { delete c; return s; }
    encode_tiled();                        // resolved outside any stream capture
    *out = c;
    return FASSMVS_OK;
}

void fassmvs_destroy(fassmvs_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    for (auto& kv : c->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto& r : c->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->pool) cudaEventDestroy(e);
    for (auto& kv : c->execs)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    for (int i = 0; i < 2; ++i) {
        if (c->host_arena[i]) cudaFreeHost(c->host_arena[i]);
        if (c->arena_ev[i]) cudaEventDestroy(c->arena_ev[i]);
        if (c->hp_in[i]) cudaEventDestroy(c->hp_in[i]);
        if (c->hp_comp[i]) cudaEventDestroy(c->hp_comp[i]);
        if (c->hp_out[i]) cudaEventDestroy(c->hp_out[i]);
    }
    if (c->hp_h2d) cudaStreamDestroy(c->hp_h2d);
    if (c->hp_d2h) cudaStreamDestroy(c->hp_d2h);
    delete c;
}

fassmvs_status fassmvs_set_config(fassmvs_ctx* c, const fassmvs_config* cfg)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    FM_TRY(check_config(c, cfg));
    c->cfg = *cfg;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_set_cameras(fassmvs_ctx* c, const double K[9], int n_nb, const double* R,
                                   const double* t, const int8_t* side)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!K || !R || !t || !side) return fail(c, FASSMVS_EINVAL, "NULL camera argument");
    if (n_nb < 1 || n_nb > fm::kMaxViews) return fail(c, FASSMVS_EINVAL, "1..%d neighbour views", fm::kMaxViews);
    double Ki[9];
    if (!k_inverse(K, Ki)) return fail(c, FASSMVS_EINVAL, "K must be upper triangular with K[2][2] = 1");
    for (int i = 0; i < 9 * n_nb; ++i)
        if (!std::isfinite(R[i])) return fail(c, FASSMVS_EINVAL, "R is not finite");
    for (int i = 0; i < 3 * n_nb; ++i)
        if (!std::isfinite(t[i])) return fail(c, FASSMVS_EINVAL, "t is not finite");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(K[i])) return fail(c, FASSMVS_EINVAL, "K is not finite");
    memcpy(c->K, K, sizeof c->K);
    c->V = n_nb;
    c->R.assign(R, R + 9 * n_nb);
    c->t.assign(t, t + 3 * n_nb);
    c->side.assign(side, side + n_nb);
    c->cams = true;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_pyramid_down(fassmvs_ctx* c, const uint8_t* in, int W, int H, uint8_t* out, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!in || !out || W < 1 || H < 1) return fail(c, FASSMVS_EINVAL, "bad pyramid arguments");
    FM_TRY(set_device(c));
    fm::launch_pyramid_down(in, W, H, W, out, (W + 1) / 2, S(stream));
    c->last = S(stream);
    return launch_status(c, "pyramid launch");
}

fassmvs_status fassmvs_census(fassmvs_ctx* c, const uint8_t* img, int W, int H, uint64_t* out, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!img || !out || W < 1 || H < 1) return fail(c, FASSMVS_EINVAL, "bad census arguments");
    FM_TRY(set_device(c));
    fm::launch_census(img, W, H, W, out, S(stream));
    c->last = S(stream);
    return launch_status(c, "census launch");
}

fassmvs_status fassmvs_cost_volume(fassmvs_ctx* c, const uint8_t* ref, const uint8_t* const* nbrs, int n_nb,
                                   const int8_t* side, int W, int H, const double K[9], const double* R,
                                   const double* t, const double n[3], double rho0, double drho, int G,
                                   const int32_t* lo, int D, int Ds, uint16_t* Sv, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    FM_TRY(set_device(c));
    c->last = S(stream);
    return cost_volume_impl(c, ref, nbrs, n_nb, side, W, H, W, K, R, t, n, rho0, drho, G, lo, D, Ds, Sv,
                            S(stream));
}

fassmvs_status fassmvs_sgm_aggregate(fassmvs_ctx* c, const uint16_t* Sv, const int32_t* lo, const int8_t* dI,
                                     const uint8_t* img, int W, int H, int D, int Ds,
                                     const fassmvs_sgm_params* prm, uint16_t* Sbar, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    FM_TRY(set_device(c));
    c->last = S(stream);
    return sgm_impl(c, Sv, lo, dI, img, W, W, H, D, Ds, prm, cost_max(c->cfg.cost) * fm::kMaxViews, Sbar,
                    S(stream));
}

fassmvs_status fassmvs_wta_refine(fassmvs_ctx* c, const uint16_t* Sbar, const int32_t* lo, int W, int H, int D,
                                  int Ds, const double K[9], const double n[3], double rho0, double drho,
                                  int G, float* depth, int32_t* gwin, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!Sbar || !K || !n || !depth || W < 1 || H < 1) return fail(c, FASSMVS_EINVAL, "bad WTA arguments");
    if (D < 1 || D > fm::kMaxSlots || Ds < D || (Ds & 7) || G < D) return fail(c, FASSMVS_EINVAL, "bad D / Ds / G");
    if (reinterpret_cast<uintptr_t>(Sbar) & 15) return fail(c, FASSMVS_EINVAL, "volume must be 16-byte aligned");
    FM_TRY(set_device(c));
    void* delta;
    FM_TRY(ensure(c, "delta_wta", sizeof(float) * (size_t)G, &delta));
    fm::launch_delta_table(rho0, drho, G, (float*)delta, S(stream));
    float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
    fm::launch_wta_refine(Sbar, lo, W, H, D, Ds, G, (const float*)delta, intr(K), nf, depth, gwin, S(stream));
    c->last = S(stream);
    return launch_status(c, "wta launch");
}

fassmvs_status fassmvs_median5(fassmvs_ctx* c, const float* in, int W, int H, float* out, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!in || !out || in == out || W < 1 || H < 1) return fail(c, FASSMVS_EINVAL, "bad median arguments");
    FM_TRY(set_device(c));
    fm::launch_median5(in, W, H, out, S(stream));
    c->last = S(stream);
    return launch_status(c, "median launch");
}

fassmvs_status fassmvs_normals(fassmvs_ctx* c, const float* depth, const uint8_t* img, int W, int H,
                               const double K[9], int radius, float beta, float* normal, float* raw,
                               const double n_plane[3], float rho_deg, float* conf, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!depth || !img || !K || !normal || W < 1 || H < 1 || radius < 0 || radius > 8 || !(beta > 0))
        return fail(c, FASSMVS_EINVAL, "bad normal arguments");
    if (conf && !n_plane) return fail(c, FASSMVS_EINVAL, "confidence needs the plane normal");
    FM_TRY(set_device(c));
    void* rawb = raw;
    if (!rawb) FM_TRY(ensure(c, "nraw", sizeof(float) * 3 * (size_t)W * H, &rawb));
    float npl[3] = {0, 0, -1};
    if (n_plane) for (int i = 0; i < 3; ++i) npl[i] = (float)n_plane[i];
    fm::launch_normals(depth, img, W, W, H, intr(K), radius, beta, (float*)rawb, normal, npl, rho_deg, conf,
                       S(stream));
    c->last = S(stream);
    return launch_status(c, "normal launch");
}

fassmvs_status fassmvs_window(fassmvs_ctx* c, const float* dc, int Wc, int Hc, int W, int H, const double K[9],
                              const double n[3], double rho0, double drho, int G, int D, int32_t* lo, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!dc || !lo || !K || !n || Wc < 1 || Hc < 1 || W < 1 || H < 1 || D < 1 || G < D)
        return fail(c, FASSMVS_EINVAL, "bad window arguments");
    FM_TRY(set_device(c));
    float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
    fm::launch_window(dc, Wc, Hc, W, H, intr(K), nf, (float)rho0, (float)drho, G, D, lo, S(stream));
    c->last = S(stream);
    return launch_status(c, "window launch");
}

fassmvs_status fassmvs_dsn(fassmvs_ctx* c, const float* dc, const float* nc, int Wc, int Hc, int W, int H,
                           const double K[9], const double n[3], double drho, int dmax, int8_t* dI, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!dc || !nc || !dI || !K || !n || Wc < 1 || Hc < 1 || W < 1 || H < 1 || dmax < 0 || dmax > 127)
        return fail(c, FASSMVS_EINVAL, "bad dsn arguments");
    FM_TRY(set_device(c));
    const float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
    fm::launch_dsn(dc, nc, Wc, Hc, W, H, intr(K), nf, (float)drho, dmax, dI, S(stream));
    c->last = S(stream);
    return launch_status(c, "dsn launch");
}

}  // extern "C"

namespace fmh {

// per-frame state of one batch call
struct FrameRun {
    const fassmvs_frame* fr;
    int V = 0, nL = 0, nR = 0, nmax = 0, P1 = 0;
    uint16_t lut[256];
    int Ws[8], Hs[8], Ps[8];
    const uint8_t* img[8][fm::kMaxViews + 1];
    float* dprev = nullptr;
    float* nprev = nullptr;
    // this level
    int w = 0, h = 0, D = 0, Ds = 0, Gl = 0;
    double Kl[9];
    double drl = 0;
    void *pS = nullptr, *pSblk = nullptr, *pSb = nullptr, *pdraw = nullptr, *pdmed = nullptr, *pnraw = nullptr, *pnrm = nullptr;
    void *plo = nullptr, *pdI = nullptr, *htab = nullptr, *delta = nullptr, *cref = nullptr;
    void* pring = nullptr;   // two-pass aggregation: rings between row blocks
};

fassmvs_status check_frame(fassmvs_ctx* c, const fassmvs_frame& f, int L, int idx)
{
    if (!f.ref || !f.nbrs || !f.K || !f.R || !f.t || !f.side || !f.depth || !f.normal || !f.conf)
        return fail(c, FASSMVS_EINVAL, "frame %d: NULL argument", idx);
    if (f.W < 2 || f.H < 2 || f.W > 8192 || f.H > 8192 || f.pitch < f.W)
        return fail(c, FASSMVS_EINVAL, "frame %d: bad size or pitch", idx);
    if (f.n_nb < 1 || f.n_nb > fm::kMaxViews) return fail(c, FASSMVS_EINVAL, "frame %d: 1..16 views", idx);
    for (int k = 0; k < f.n_nb; ++k)
        if (!f.nbrs[k]) return fail(c, FASSMVS_EINVAL, "frame %d: neighbour %d is NULL", idx, k);
    double Ki[9];
    if (!k_inverse(f.K, Ki)) return fail(c, FASSMVS_EINVAL, "frame %d: K must be upper triangular", idx);
    for (int i = 0; i < 9 * f.n_nb; ++i)
        if (!std::isfinite(f.R[i])) return fail(c, FASSMVS_EINVAL, "frame %d: R is not finite", idx);
    for (int i = 0; i < 3 * f.n_nb; ++i)
        if (!std::isfinite(f.t[i])) return fail(c, FASSMVS_EINVAL, "frame %d: t is not finite", idx);
    if (((f.W - 1) >> (L - 1)) + 1 < 2 || ((f.H - 1) >> (L - 1)) + 1 < 2)
        return fail(c, FASSMVS_EINVAL, "frame %d: image too small for %d levels", idx, L);
    if (f.planes.G0 < 1) return fail(c, FASSMVS_EINVAL, "frame %d: G0 must be >= 1", idx);
    if ((f.planes.G0 - 1) / (1 << (L - 1)) + 1 > fm::kMaxSlots)
        return fail(c, FASSMVS_EINVAL, "frame %d: top level has more than 256 planes (Sec. 3.2 cap)", idx);
    if (!(std::isfinite(f.planes.rho_far) && std::isfinite(f.planes.drho)) ||
        !(f.planes.rho_far > 0.0 || (f.planes.rho_far >= 0.0 && f.planes.drho > 0.0)))
        return fail(c, FASSMVS_EINVAL, "frame %d: plane list must have positive inverse distances", idx);
    return FASSMVS_OK;
}


std::string fname(int f, const char* what)
{
    char b[48];
    snprintf(b, sizeof b, "f%d:%s", f, what);
    return b;
}

// control words of the two-pass aggregation of up to kWaveBatch frames: the
// two passes' tickets, then per frame its flags (fm::wave_flag_bytes of the
// tallest frame the checks allow)
constexpr size_t kWaveCtlHead = 256;
constexpr size_t kWaveCtlFrame = 2 * 2 * 1024 * sizeof(int);
constexpr size_t kWaveCtlBytes = kWaveCtlHead + fm::kWaveBatch * kWaveCtlFrame;

void frame_scratch_layout(const fassmvs_config& cfg, int W, int H, int V, int G0, int parts, int wave_cap,
                          std::vector<std::pair<std::string, size_t>>& out)
{
    std::map<std::string, size_t> m;
    auto need = [&](const char* name, size_t b) { m[name] = std::max(m[name], b); };
    const int L = cfg.levels;
    int w = W, h = H;
    for (int l = 0; l < L; ++l) {
        if (l > 0) { w = (w + 1) / 2; h = (h + 1) / 2; }
        const size_t np = (size_t)w * h;
        const int Gl = (G0 - 1) / (1 << l) + 1;
        const int D = (l == L - 1) ? Gl : std::min(cfg.D[l], Gl);
        const size_t Ds = (size_t)((D + 15) & ~15);
        need("S", 2 * np * Ds);
        need("Sblk", 2 * np * Ds);
        if (parts > 0) need("Sbar", 2 * np * Ds * parts);
        else need("wring", fm::wave_ring_bytes(w, h, wave_cap, nullptr));
        need("draw", 4 * np);
        need("nraw", 12 * np);
        need("cref", 8 * np);
        need("htab", 72 * (size_t)Gl * V);
        need("delta", 4 * (size_t)Gl);
        if (l > 0) {
            need((l & 1) ? "dmedA" : "dmedB", 4 * np);
            need((l & 1) ? "nrmA" : "nrmB", 12 * np);
        }
        if (l < L - 1) need("lo", 4 * np);
        if (cfg.variant == 1) need("dI", 8 * np);
    }
    out.assign(m.begin(), m.end());
}

// grows both pinned staging halves to at least `bytes` now
fassmvs_status stage_reserve(fassmvs_ctx* c, size_t bytes)
{
    if (bytes <= c->host_cap) return FASSMVS_OK;
    for (int i = 0; i < 2; ++i) {
        if (c->arena_ev[i]) FM_TRY(cuda_check(c, cudaEventSynchronize(c->arena_ev[i]), "staging wait"));
        if (c->host_arena[i]) cudaFreeHost(c->host_arena[i]);
        c->host_arena[i] = nullptr;
        FM_TRY(cuda_check(c, cudaHostAlloc((void**)&c->host_arena[i], bytes, cudaHostAllocDefault), "cudaHostAlloc"));
        if (!c->arena_ev[i])
            FM_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->arena_ev[i], cudaEventDisableTiming), "event"));
    }
    c->host_cap = bytes;
    return FASSMVS_OK;
}

fassmvs_status ctx_reserve(fassmvs_ctx* c, size_t bytes)
{
    void* p;
    FM_TRY(stage_reserve(c, bytes));
    FM_TRY(ensure(c, "stageA", bytes, &p));
    FM_TRY(ensure(c, "stageB", bytes, &p));
    FM_TRY(ensure(c, "counter", 256, &p));
    FM_TRY(ensure(c, "wave_ctl", kWaveCtlBytes, &p));
    for (const char* name : {"cost_err", "sgm_err"}) {
        const bool fresh = !c->bufs.count(name);
        FM_TRY(ensure(c, name, sizeof(int), &p));
        if (fresh) FM_TRY(cuda_check(c, cudaMemset(p, 0, sizeof(int)), "memset"));
    }
    return FASSMVS_OK;
}

// scratch buffer `name` of frame f of the batch
fassmvs_status fscratch(fassmvs_ctx* c, int f, const char* name, size_t bytes, void** out)
{
    if (c->scratch_fn) return c->scratch_fn(c->scratch_user, f, name, bytes, out);
    return ensure(c, fname(f, name).c_str(), bytes, out);
}

// partial sums of the per-direction aggregation: one per direction when
// automatic (and for the two-pass form's fallback)
int sgm_parts(const fassmvs_tuning& t, int paths)
{
    const int p = t.sgm_parts > 0 ? t.sgm_parts : paths;
    return p > paths ? paths : p;
}

int agg_parts(const fassmvs_tuning& t, int paths, int device)
{
    if (t.sgm_parts == kSgmTwoPass && fm::wave_capacity(device) > 0) return 0;
    return sgm_parts(t, paths);
}

// Picks the staging half for one call and waits until the call that last used
// it has finished on the device; grows both halves (pinned host and device
// mirror) when the batch needs more.  Never runs while a stream is captured.
fassmvs_status stage_prepare(fassmvs_ctx* c, const fassmvs_frame* frames, int n, int chunk_planes, Stage* out)
{
    const int L = c->cfg.levels;
    const int cmin = chunk_planes > 0 ? chunk_planes : 8;   // automatic chunks hold >= 8 planes
    size_t need = 4096;
    for (int l = 0; l < L; ++l) {
        size_t items = 0;
        for (int f = 0; f < n; ++f) {
            const int w = ((frames[f].W - 1) >> l) + 1, h = ((frames[f].H - 1) >> l) + 1;
            items += (size_t)fm::cost_tiles_x(w) * fm::cost_tiles_y(h) *
                     ((fm::kMaxSlots + cmin - 1) / cmin + 1);
        }
        need += 2 * 256 + n * sizeof(fm::CostArgs) + items * sizeof(int4) +
                n * (256 + sizeof(CUtensorMap) * (size_t)fm::kMaxViews);
    }
    FM_TRY(stage_reserve(c, need));
    const int half = c->arena_half;
    c->arena_half ^= 1;
    FM_TRY(cuda_check(c, cudaEventSynchronize(c->arena_ev[half]), "staging wait"));
    void* dstage;
    // the device mirror follows this call's need (the host halves may be
    // reserved larger)
    FM_TRY(ensure(c, half ? "stageB" : "stageA", need, &dstage));
    *out = Stage{c->host_arena[half], (unsigned char*)dstage, 0, need, half};
    return FASSMVS_OK;
}

fassmvs_status run_batch(fassmvs_ctx* c, const fassmvs_frame* frames, int n, cudaStream_t st,
                         const fassmvs_tuning& tn, const Stage& stage, const fm::PyrSet* pyrs)
{
    const fassmvs_config& cfg = c->cfg;
    const int L = cfg.levels;
    const int chunk_planes = tn.chunk_planes, ctas_per_sm = tn.ctas_per_sm;
    const int parts = agg_parts(tn, cfg.paths, c->device);   // 0: two-pass form
    const int wave_cap = parts == 0 ? fm::wave_capacity(c->device) : 0;
    const bool capturing = [&] {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        return cs != cudaStreamCaptureStatusNone;
    }();
    const bool prof = c->prof;
    if (capturing) c->prof = false;
    struct Restore { fassmvs_ctx* c; bool p; ~Restore() { c->prof = p; } } restore{c, prof};

    std::vector<FrameRun> fr(n);
    for (int f = 0; f < n; ++f) {
        FrameRun& F = fr[f];
        F.fr = &frames[f];
        F.V = frames[f].n_nb;
        for (int k = 0; k < F.V; ++k) { if (frames[f].side[k] < 0) ++F.nL; else ++F.nR; }
        F.nmax = std::max(F.nL, F.nR);
        F.P1 = cfg.p1 * F.nmax;
        p2_table(F.P1, cfg.alpha, cfg.beta, F.lut);
        F.Ws[0] = frames[f].W; F.Hs[0] = frames[f].H; F.Ps[0] = frames[f].pitch;
        F.img[0][0] = frames[f].ref;
        for (int k = 0; k < F.V; ++k) F.img[0][k + 1] = frames[f].nbrs[k];
        for (int l = 1; l < L; ++l) {
            F.Ws[l] = (F.Ws[l - 1] + 1) / 2;
            F.Hs[l] = (F.Hs[l - 1] + 1) / 2;
            F.Ps[l] = (F.Ws[l] + 15) & ~15;    // 16-byte rows: the cost kernel stages them by TMA
        }
        if (pyrs) {
            // resident pyramids (serving form): level l of view k, pitch W_l
            for (int l = 0; l < L; ++l) {
                if (l > 0) F.Ps[l] = pyrs[f].pitch[l];
                for (int k = 0; k <= F.V; ++k) F.img[l][k] = pyrs[f].img[l][k];
            }
        }
    }
    void* counter;
    FM_TRY(ensure(c, "counter", 256, &counter));
    // raised by the cost kernel when a staged copy misses its bound (read by fassmvs_sync)
    void* cost_err;
    const bool fresh_err = !c->bufs.count("cost_err");
    FM_TRY(ensure(c, "cost_err", sizeof(int), &cost_err));
    if (fresh_err) FM_TRY(cuda_check(c, cudaMemsetAsync(cost_err, 0, sizeof(int), st), "memset"));
    // the two-pass aggregation's control words and its error word (a row
    // whose wait on a neighbouring row gave up; read by fassmvs_sync)
    void *wave_ctl = nullptr, *sgm_err = nullptr;
    if (parts == 0) {
        FM_TRY(ensure(c, "wave_ctl", kWaveCtlBytes, &wave_ctl));
        const bool fresh = !c->bufs.count("sgm_err");
        FM_TRY(ensure(c, "sgm_err", sizeof(int), &sgm_err));
        if (fresh) FM_TRY(cuda_check(c, cudaMemsetAsync(sgm_err, 0, sizeof(int), st), "memset"));
    }
    static thread_local fm::WaveBatch wb;      // 12 KB: kept off the stack
    Stage sg = stage;
    std::vector<fm::SgmArgs> sargs;
    static thread_local fm::SgmBatch sb;       // 20 KB: kept off the stack

    // ---- pyramids of every frame
    if (!pyrs) {
        StageTimer tm(c, FASSMVS_STAGE_PYRAMID, st);
        for (int f = 0; f < n; ++f) {
            FrameRun& F = fr[f];
            for (int l = 1; l < L; ++l) {
                void* p;
                FM_TRY(fscratch(c, f, ("pyr" + std::to_string(l)).c_str(), (size_t)(F.V + 1) * F.Ps[l] * F.Hs[l], &p));
                for (int k = 0; k <= F.V; ++k) {
                    uint8_t* o = (uint8_t*)p + (size_t)k * F.Ps[l] * F.Hs[l];
                    fm::launch_pyramid_down(F.img[l - 1][k], F.Ws[l - 1], F.Hs[l - 1], F.Ps[l - 1], o, F.Ps[l], st);
                    F.img[l][k] = o;
                }
            }
        }
    }
    // persistent cost CTAs (0: one short-lived CTA per work item); the
    // automatic plane chunking aims at three waves of two CTAs per SM either way
    int ctas = 0, wave = 0;
    {
        int nsm = 148;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
        ctas = nsm * ctas_per_sm;
        wave = nsm * (ctas_per_sm ? ctas_per_sm : 2);
    }
    for (int l = L - 1; l >= 0; --l) {
        char level_name[32];
        snprintf(level_name, sizeof level_name, "fassmvs level %d", l);
        NvtxRange level_range(level_name);
        const size_t block0 = (sg.off + 255) & ~(size_t)255;
        size_t at_cargs, at_items;
        fm::CostArgs* cargs = (fm::CostArgs*)sg.take(sizeof(fm::CostArgs) * n, at_cargs);
        if (!cargs) return fail(c, FASSMVS_EINTERNAL, "staging overflow");
        sargs.resize(n);
        std::vector<int4> items;
        std::vector<int> order(n);
        for (int f = 0; f < n; ++f) {
            FrameRun& F = fr[f];
            const fassmvs_frame& X = *F.fr;
            F.w = F.Ws[l]; F.h = F.Hs[l];
            const size_t np = (size_t)F.w * F.h;
            const double sc = (double)(1 << l);
            const double Kl[9] = {X.K[0] / sc, X.K[1] / sc, X.K[2] / sc, 0.0, X.K[4] / sc, X.K[5] / sc, 0.0, 0.0, 1.0};
            memcpy(F.Kl, Kl, sizeof Kl);
            F.Gl = (X.planes.G0 - 1) / (1 << l) + 1;
            F.drl = X.planes.drho * sc;
            F.D = (l == L - 1) ? F.Gl : std::min(cfg.D[l], F.Gl);
            F.Ds = (F.D + 15) & ~15;          // whole 16-plane blocks
            FM_TRY(fscratch(c, f, "S", sizeof(uint16_t) * np * F.Ds, &F.pS));
            FM_TRY(fscratch(c, f, "Sblk", sizeof(uint16_t) * np * F.Ds, &F.pSblk));
            if (parts > 0) FM_TRY(fscratch(c, f, "Sbar", sizeof(uint16_t) * np * F.Ds * parts, &F.pSb));
            else FM_TRY(fscratch(c, f, "wring", fm::wave_ring_bytes(F.w, F.h, wave_cap, nullptr), &F.pring));
            FM_TRY(fscratch(c, f, "draw", sizeof(float) * np, &F.pdraw));
            FM_TRY(fscratch(c, f, "nraw", sizeof(float) * 3 * np, &F.pnraw));
            FM_TRY(fscratch(c, f, "cref", sizeof(uint64_t) * np, &F.cref));
            FM_TRY(fscratch(c, f, "htab", sizeof(float) * 18 * (size_t)F.Gl * F.V, &F.htab));
            FM_TRY(fscratch(c, f, "delta", sizeof(float) * (size_t)F.Gl, &F.delta));
            if (l > 0) {
                FM_TRY(fscratch(c, f, (l & 1) ? "dmedA" : "dmedB", sizeof(float) * np, &F.pdmed));
                FM_TRY(fscratch(c, f, (l & 1) ? "nrmA" : "nrmB", sizeof(float) * 3 * np, &F.pnrm));
            } else {
                F.pdmed = X.depth;
                F.pnrm = X.normal;
            }
            F.plo = nullptr;
            F.pdI = nullptr;
            if (l < L - 1) FM_TRY(fscratch(c, f, "lo", sizeof(int32_t) * np, &F.plo));
            if (cfg.variant == 1) FM_TRY(fscratch(c, f, "dI", 8 * np, &F.pdI));
            const float nf[3] = {(float)X.planes.n[0], (float)X.planes.n[1], (float)X.planes.n[2]};
            if (l < L - 1) {
                StageTimer tm(c, FASSMVS_STAGE_WINDOW, st);
                fm::launch_window(F.dprev, F.Ws[l + 1], F.Hs[l + 1], F.w, F.h, intr(F.Kl), nf, (float)X.planes.rho_far,
                                  (float)F.drl, F.Gl, F.D, (int32_t*)F.plo, st);
                if (cfg.variant == 1)
                    fm::launch_dsn(F.dprev, F.nprev, F.Ws[l + 1], F.Hs[l + 1], F.w, F.h, intr(F.Kl), nf,
                                   (float)F.drl, cfg.dmax, (int8_t*)F.pdI, st);
            } else if (cfg.variant == 1) {
                FM_TRY(cuda_check(c, cudaMemsetAsync(F.pdI, 0, 8 * np, st), "memset dI"));
            }
            fm::ViewGeom vg;
            FM_TRY(view_geom(c, F.Kl, F.V, X.R, X.t, X.planes.n, &vg));
            fm::LevelPlanes lp{X.planes.rho_far, F.drl, F.Gl, F.V, 0.5 * (F.w - 1), 0.5 * (F.h - 1)};
            {
                StageTimer tm(c, FASSMVS_STAGE_CENSUS, st);
                fm::launch_prep_level(vg, lp, (float*)F.htab, (float*)F.delta, st);
                fm::launch_census(F.img[l][0], F.w, F.h, F.Ps[l], (uint64_t*)F.cref, st);
            }
            // cost arguments
            fm::CostArgs& a = cargs[f];
            memset(&a, 0, sizeof a);
            a.cost = cfg.cost;
            a.ref = F.img[l][0];
            a.ref_pitch = F.Ps[l];
            a.cref = (const uint64_t*)F.cref;
            for (int k = 0; k < F.V; ++k) {
                a.views.img[k] = F.img[l][k + 1];
                a.views.side[k] = X.side[k] < 0 ? -1 : 1;
            }
            a.V = F.V; a.W = F.w; a.H = F.h; a.pitch = F.Ps[l];
            a.nL = F.nL; a.nR = F.nR; a.nmax = F.nmax;
            a.mL = F.nL ? ((1ull << 32) + F.nL - 1) / F.nL : 0;
            a.mR = F.nR ? ((1ull << 32) + F.nR - 1) / F.nR : 0;
            a.htab = (const float*)F.htab;
            a.lo = (const int32_t*)F.plo;
            a.D = F.D; a.Ds = F.Ds; a.G = F.Gl;
            // the cost kernel writes 16-plane blocks [Ds / 16][h][w][16]: its
            // per-plane 2-byte stores then complete their 32-byte sectors within
            // 16 planes (with [h][w][Ds] an L2 line stays open over 64 planes
            // and the ~110 MB of open lines of the resident CTAs thrash the
            // L2); a relayout gives the aggregation [h][w][Ds]
            a.pstride = 16;
            a.bstride = 16 * np;
            a.bshift = 4;
            a.S = (uint16_t*)F.pSblk;
            // tensor maps of the views for the kernel's staging (all views or none)
            {
                size_t at_tm;
                unsigned char* tm = (unsigned char*)sg.take(sizeof(CUtensorMap) * (size_t)F.V, at_tm);
                if (!tm) return fail(c, FASSMVS_EINTERNAL, "staging overflow");
                bool all = true;
                for (int k = 0; k < F.V && all; ++k)
                    all = encode_view(tm + sizeof(CUtensorMap) * k, F.img[l][k + 1], F.w, F.h, F.Ps[l]);
                a.tmaps = (all && !tn.no_staging) ? (const void*)(sg.dev + at_tm) : nullptr;
            }
            a.err = (int*)cost_err;
            a.stage_test = c->inject == 1;
            if (f == 0 && l == c->dbg_level && c->dbg_warp_g >= 0) {
                // the warped values of one (plane, view) pair; NaN where no tile sampled it
                void* p;
                FM_TRY(ensure(c, "dbg:warp", sizeof(float) * np, &p));
                FM_TRY(cuda_check(c, cudaMemsetAsync(p, 0xFF, sizeof(float) * np, st), "capture"));
                a.dbg_warp = (float*)p;
                a.dbg_g = c->dbg_warp_g;
                a.dbg_k = c->dbg_warp_k;
            }
            // aggregation arguments
            fm::SgmArgs& g = sargs[f];
            memset(&g, 0, sizeof g);
            int p2max = cfg.adaptive_p2 ? 0 : cfg.p2 * F.nmax;
            if (cfg.adaptive_p2) {
                g.use_lut = 1;
                for (int i = 0; i < 256; ++i) { g.lut[i] = F.lut[i]; p2max = std::max(p2max, (int)F.lut[i]); }
            }
            p2max = std::max(p2max, F.P1);
            if ((long long)cfg.paths * (cost_max(cfg.cost) * F.nmax + p2max) >= 65536)
                return fail(c, FASSMVS_EINVAL, "frame %d: aggregated costs could exceed 16 bits", f);
            g.S = (const uint16_t*)F.pS; g.lo = (const int32_t*)F.plo; g.dI = (const int8_t*)F.pdI;
            g.img = F.img[l][0]; g.img_pitch = F.Ps[l];
            g.W = F.w; g.H = F.h; g.D = F.D; g.Ds = F.Ds;
            g.pstride = (size_t)F.Ds;
            g.bstride = 8;
            g.bshift = 3;
            g.paths = cfg.paths; g.variant = cfg.variant; g.p1 = F.P1; g.p2 = cfg.p2 * F.nmax; g.dmax = cfg.dmax;
            g.Sbar = (uint16_t*)F.pSb;
            g.part_stride = np * F.Ds;
            order[f] = f;
        }
        // cost work items: larger views x window first, frame by frame
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            return (long long)fr[x].V * fr[x].D * fr[x].w * fr[x].h > (long long)fr[y].V * fr[y].D * fr[y].w * fr[y].h;
        });
        // plane chunks per tile: fixed size, or (automatic) at least about
        // three waves of the persistent CTAs, chunks of at least 8 planes
        long long tiles = 0;
        for (int f = 0; f < n; ++f) tiles += (long long)fm::cost_tiles_x(fr[f].w) * fm::cost_tiles_y(fr[f].h);
        const int auto_nz = (int)std::max(1LL, (3LL * wave + tiles - 1) / tiles);
        // automatic: from auto_nz up to twice that (chunks of >= 8 planes), the
        // count whose items fill their last wave of persistent CTAs best
        auto fill = [&](long long items) {
            const long long w = (items + wave - 1) / wave;
            return (double)items / (double)(w * wave);
        };
        int best_nz = auto_nz;
        {
            int dmax = 1;
            for (int f = 0; f < n; ++f) dmax = std::max(dmax, fr[f].D);
            const int hi = std::max(1, std::min(2 * auto_nz, (dmax + 7) / 8));
            double bf = -1.0;
            for (int z = std::min(auto_nz, hi); z <= hi; ++z) {
                const double q = fill(tiles * z);
                if (q > bf + 0.02) { bf = q; best_nz = z; }
            }
        }
        for (int f : order) {
            const FrameRun& F = fr[f];
            const int nz = chunk_planes > 0 ? std::max(1, (F.D + chunk_planes - 1) / chunk_planes)
                                            : std::max(1, std::min(best_nz, (F.D + 7) / 8));
            const int tx = fm::cost_tiles_x(F.w), ty = fm::cost_tiles_y(F.h);
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ty; ++y)
                    for (int x = 0; x < tx; ++x) items.push_back(make_int4(f, x, y, z | (nz << 16)));
        }
        int4* hitems = (int4*)sg.take(sizeof(int4) * items.size(), at_items);
        if (!hitems) return fail(c, FASSMVS_EINTERNAL, "staging overflow");
        memcpy(hitems, items.data(), sizeof(int4) * items.size());
        FM_TRY(cuda_check(c, cudaMemcpyAsync(sg.dev + block0, sg.host + block0, sg.off - block0, cudaMemcpyHostToDevice, st),
                          "staging copy"));
        {
            StageTimer tm(c, FASSMVS_STAGE_COST, st);
            // the kernel that copies the warped tile out only while a pair is chosen
            const bool dbg = l == c->dbg_level && c->dbg_warp_g >= 0;
            fm::launch_cost_batch((const fm::CostArgs*)(sg.dev + at_cargs), (const int4*)(sg.dev + at_items),
                                  (int)items.size(), (int*)counter, ctas, cfg.cost != 0, dbg, st);
        }
        {
            StageTimer tm(c, FASSMVS_STAGE_RELAYOUT, st);
            for (int f = 0; f < n; ++f)
                fm::launch_relayout16((const uint16_t*)fr[f].pSblk, (uint16_t*)fr[f].pS, (size_t)fr[f].w * fr[f].h,
                                      fr[f].Ds, st);
        }
        // debug capture of frame 0 at the selected level: the cost volume,
        // the window starts and the surface-normal jumps
        const bool dbg = l == c->dbg_level;
        if (dbg) {
            const FrameRun& F = fr[0];
            const size_t np = (size_t)F.w * F.h;
            const int dims[5] = {F.w, F.h, F.D, F.Ds, F.Gl};
            memcpy(c->dbg_dims, dims, sizeof dims);
            void* p;
            FM_TRY(ensure(c, "dbg:S", 2 * np * F.Ds, &p));
            FM_TRY(cuda_check(c, cudaMemcpyAsync(p, F.pS, 2 * np * F.Ds, cudaMemcpyDeviceToDevice, st), "capture"));
            FM_TRY(ensure(c, "dbg:lo", 4 * np, &p));
            FM_TRY(cuda_check(c, F.plo ? cudaMemcpyAsync(p, F.plo, 4 * np, cudaMemcpyDeviceToDevice, st)
                                       : cudaMemsetAsync(p, 0, 4 * np, st), "capture"));
            FM_TRY(ensure(c, "dbg:dI", 8 * np, &p));
            FM_TRY(cuda_check(c, F.pdI ? cudaMemcpyAsync(p, F.pdI, 8 * np, cudaMemcpyDeviceToDevice, st)
                                       : cudaMemsetAsync(p, 0, 8 * np, st), "capture"));
        }
        void *dbg_gwin = nullptr, *dbg_agg = nullptr;
        if (dbg) {
            const FrameRun& F = fr[0];
            FM_TRY(ensure(c, "dbg:agg", 2 * (size_t)F.w * F.h * F.Ds, &dbg_agg));
            FM_TRY(ensure(c, "dbg:gwin", 4 * (size_t)F.w * F.h, &dbg_gwin));
        }
        if (parts == 0) {
            StageTimer tm(c, FASSMVS_STAGE_SGM, st);
            // the two-pass form over groups of up to kWaveBatch frames; pass B
            // takes the winner and writes the depth, so no winner-takes-all
            // launch follows
            for (int f0 = 0; f0 < n; f0 += fm::kWaveBatch) {
                const int m = std::min(n - f0, fm::kWaveBatch);
                FM_TRY(cuda_check(c, cudaMemsetAsync(wave_ctl, 0, kWaveCtlHead + m * kWaveCtlFrame, st), "memset"));
                wb.nframes = m;
                wb.ticket = (int*)wave_ctl;
                wb.err = (int*)sgm_err;
                int items = 0;
                for (int i = 0; i < m; ++i) {
                    const int f = f0 + i;
                    const FrameRun& F = fr[f];
                    const fassmvs_frame& X = *F.fr;
                    fm::WaveFrame& Wf = wb.f[i];
                    Wf.a = sargs[f];
                    Wf.a.Sbar = dbg && f == 0 ? (uint16_t*)dbg_agg : nullptr;
                    Wf.T1 = (uint16_t*)F.pSblk;   // the blocked volume is dead after the relayout
                    Wf.delta = (const float*)F.delta;
                    Wf.G = F.Gl;
                    Wf.K = intr(F.Kl);
                    Wf.n0 = (float)X.planes.n[0];
                    Wf.n1 = (float)X.planes.n[1];
                    Wf.n2 = (float)X.planes.n[2];
                    Wf.depth = cfg.median5 ? (float*)F.pdraw : (float*)F.pdmed;
                    Wf.gwin = dbg && f == 0 ? (int32_t*)dbg_gwin : nullptr;
                    size_t scal_off = 0;
                    fm::wave_ring_bytes(F.w, F.h, wave_cap, &scal_off);
                    Wf.gring = (uint4*)F.pring;
                    Wf.gscal = (int4*)((char*)F.pring + scal_off);
                    Wf.ring = fm::wave_ring_cols(F.w, F.h, wave_cap);
                    Wf.gflag = (int*)((char*)wave_ctl + kWaveCtlHead + i * kWaveCtlFrame);
                    Wf.nblocks = fm::wave_blocks(F.h);
                    wb.item0[i] = items;
                    items += Wf.nblocks;
                }
                wb.item0[m] = items;
                const int ctas = std::min(wave_cap, items);
                fm::launch_sgm_wave(wb, 0, ctas, st);
                fm::launch_sgm_wave(wb, 1, ctas, st);
            }
        } else {
            StageTimer tm(c, FASSMVS_STAGE_SGM, st);
            // `parts` partial sums: launch g runs, for every part k, direction
            // k * (paths / parts) + g into part k (writing it when g == 0), so
            // `parts` directions run concurrently; frames in groups of up to
            // kSgmBatch, each group's arguments by value
            const int per = cfg.paths / parts;
            for (int f0 = 0; f0 < n; f0 += fm::kSgmBatch) {
                const int m = std::min(n - f0, fm::kSgmBatch);
                sb.nframes = m;
                for (int f = 0; f < m; ++f) sb.a[f] = sargs[f0 + f];
                for (int g = 0; g < per; ++g) {
                    // slots with the longest paths first (they start in the first wave)
                    int order_k[8];
                    for (int k = 0; k < parts; ++k) order_k[k] = k;
                    auto plen = [&](int k) {
                        int dx, dy;
                        fm::sgm_dir_of(k * per + g, &dx, &dy);
                        return dy == 0 ? 2 : (dx == 0 ? 1 : 0);
                    };
                    std::stable_sort(order_k, order_k + parts, [&](int x, int y) { return plen(x) > plen(y); });
                    sb.nslots = parts;
                    int acc = 0;
                    for (int j = 0; j < parts; ++j) {
                        const int k = order_k[j], r = k * per + g;
                        sb.r[j] = r;
                        fm::sgm_dir_of(r, &sb.dx[j], &sb.dy[j]);
                        sb.part[j] = k;
                        sb.first[j] = g == 0;
                        for (int f = 0; f < m; ++f) {
                            sb.seg[j][f] = acc;
                            acc += fm::sgm_lines(fr[f0 + f].w, fr[f0 + f].h, r);
                        }
                        sb.seg[j][m] = acc;
                    }
                    fm::launch_sgm_batch(sb, st);
                }
            }
        }
        if (dbg && parts > 0) {
            const FrameRun& F = fr[0];
            const size_t nv = (size_t)F.w * F.h * F.Ds;
            fm::launch_sum_parts((const uint16_t*)F.pSb, parts, nv, nv, (uint16_t*)dbg_agg, st);
        }
        for (int f = 0; f < n; ++f) {
            FrameRun& F = fr[f];
            const fassmvs_frame& X = *F.fr;
            const float nf[3] = {(float)X.planes.n[0], (float)X.planes.n[1], (float)X.planes.n[2]};
            if (parts > 0) {
                StageTimer tm(c, FASSMVS_STAGE_WTA, st);
                fm::launch_wta_refine((const uint16_t*)F.pSb, (const int32_t*)F.plo, F.w, F.h, F.D, F.Ds, F.Gl,
                                      (const float*)F.delta, intr(F.Kl), nf,
                                      cfg.median5 ? (float*)F.pdraw : (float*)F.pdmed,
                                      dbg && f == 0 ? (int32_t*)dbg_gwin : nullptr, st, parts,
                                      (size_t)F.w * F.h * F.Ds);
            }
            if (cfg.median5) {
                StageTimer tm(c, FASSMVS_STAGE_MEDIAN, st);
                fm::launch_median5((const float*)F.pdraw, F.w, F.h, (float*)F.pdmed, st);
            }
            if (dbg && f == 0) {
                const size_t np = (size_t)F.w * F.h;
                void* p;
                FM_TRY(ensure(c, "dbg:draw", 4 * np, &p));
                FM_TRY(cuda_check(c, cudaMemcpyAsync(p, cfg.median5 ? F.pdraw : F.pdmed, 4 * np,
                                                     cudaMemcpyDeviceToDevice, st), "capture"));
                FM_TRY(ensure(c, "dbg:dmed", 4 * np, &p));
                FM_TRY(cuda_check(c, cudaMemcpyAsync(p, F.pdmed, 4 * np, cudaMemcpyDeviceToDevice, st), "capture"));
            }
            {
                StageTimer tm(c, FASSMVS_STAGE_NORMALS, st);
                fm::launch_normals((const float*)F.pdmed, F.img[l][0], F.Ps[l], F.w, F.h, intr(F.Kl), cfg.normal_radius,
                                   cfg.normal_beta, (float*)F.pnraw, (float*)F.pnrm, nf, cfg.rho_deg,
                                   l == 0 ? X.conf : nullptr, st);
            }
            if (dbg && f == 0) {
                void* p;
                FM_TRY(ensure(c, "dbg:nrm", 12 * (size_t)F.w * F.h, &p));
                FM_TRY(cuda_check(c, cudaMemcpyAsync(p, F.pnrm, 12 * (size_t)F.w * F.h, cudaMemcpyDeviceToDevice, st),
                                  "capture"));
            }
            F.dprev = (float*)F.pdmed;
            F.nprev = (float*)F.pnrm;
        }
        FM_TRY(launch_status(c, "level launch"));
    }
    FM_TRY(cuda_check(c, cudaEventRecordWithFlags(c->arena_ev[sg.half], st, capturing ? cudaEventRecordExternal : 0),
                      "staging event"));
    return FASSMVS_OK;
}

uint64_t batch_signature(const fassmvs_ctx* c, const fassmvs_frame* fr, int n, const fassmvs_tuning* tn)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)n);
    if (tn) {
        mix((uint64_t)tn->chunk_planes); mix((uint64_t)tn->ctas_per_sm); mix((uint64_t)tn->sgm_parts);
        mix((uint64_t)tn->no_staging);
    }
    const unsigned char* cb = reinterpret_cast<const unsigned char*>(&c->cfg);
    for (size_t i = 0; i < sizeof(c->cfg); ++i) mix(cb[i]);
    for (int f = 0; f < n; ++f) {
        mix((uint64_t)fr[f].W); mix((uint64_t)fr[f].H); mix((uint64_t)fr[f].pitch);
        mix((uint64_t)fr[f].n_nb); mix((uint64_t)fr[f].planes.G0);
    }
    return h;
}

fassmvs_status check_tuning(fassmvs_ctx* c, const fassmvs_tuning& t)
{
    if (t.chunk_planes < 0 || t.chunk_planes > 256 || t.ctas_per_sm < 0 || t.ctas_per_sm > 2)
        return fail(c, FASSMVS_EINVAL, "chunk_planes 0 (automatic) or 1..256, ctas_per_sm 0 (one CTA per item), 1 or 2");
    if (t.sgm_parts != 0 && t.sgm_parts != kSgmTwoPass && t.sgm_parts != 1 && t.sgm_parts != 2 &&
        t.sgm_parts != 4 && t.sgm_parts != 8)
        return fail(c, FASSMVS_EINVAL, "sgm_parts 0 (automatic), -1 (two-pass), 1, 2, 4 or 8");
    if (t.no_staging != 0 && t.no_staging != 1) return fail(c, FASSMVS_EINVAL, "no_staging 0 or 1");
    return FASSMVS_OK;
}

fassmvs_status estimate_batch_impl(fassmvs_ctx* c, const fassmvs_frame* frames, int n, cudaStream_t st)
{
    if (n < 1 || n > 64) return fail(c, FASSMVS_EINVAL, "1..64 frames per batch");
    if (!frames) return fail(c, FASSMVS_EINVAL, "frames is NULL");
    for (int f = 0; f < n; ++f) FM_TRY(check_frame(c, frames[f], c->cfg.levels, f));
    FM_TRY(set_device(c));
    c->last = st;
    fassmvs_tuning tn = c->tune;
    auto it = c->tuned.find(batch_signature(c, frames, n, nullptr));
    if (it != c->tuned.end()) tn = it->second;
    const uint64_t sig = batch_signature(c, frames, n, &tn);
    Stage sg;
    FM_TRY(stage_prepare(c, frames, n, tn.chunk_planes, &sg));
    if (!c->graph || st == nullptr || !c->seen.count(sig) || c->dbg_level >= 0) {
        // eager (and the first run of a shape: allocates all scratch)
        FM_TRY(run_batch(c, frames, n, st, tn, sg, nullptr));
        c->seen[sig] = 1;
        return FASSMVS_OK;
    }
    FM_TRY(cuda_check(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin capture"));
    fassmvs_status rs = run_batch(c, frames, n, st, tn, sg, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rs != FASSMVS_OK) { if (g) cudaGraphDestroy(g); return rs; }
    FM_TRY(cuda_check(c, ce, "end capture"));
    cudaGraphExec_t& ex = c->execs[sig];
    if (ex) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(ex);
            ex = nullptr;
        }
    }
    if (!ex) {
        cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        if (ie != cudaSuccess) { cudaGraphDestroy(g); ex = nullptr; return cuda_check(c, ie, "graph instantiate"); }
    }
    cudaGraphDestroy(g);
    return cuda_check(c, cudaGraphLaunch(ex, st), "graph launch");
}

// Alg. 3 weights: a 7-tap Gaussian of sigma 1.4, quantised to integers that
// sum to 256 (the rounding remainder goes to the centre tap)
fm::DogWeights dog_weights()
{
    fm::DogWeights w;
    double g[7], sum = 0.0;
    for (int i = 0; i < 7; ++i) {
        g[i] = std::exp(-(double)((i - 3) * (i - 3)) / (2.0 * 1.4 * 1.4));
        sum += g[i];
    }
    int tot = 0;
    for (int i = 0; i < 7; ++i) {
        w.w[i] = (int32_t)std::floor(256.0 * g[i] / sum + 0.5);
        tot += w.w[i];
    }
    w.w[3] += 256 - tot;
    return w;
}

}  // namespace fmh

extern "C" {

fassmvs_status fassmvs_estimate_batch(fassmvs_ctx* c, const fassmvs_frame* frames, int n, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    return estimate_batch_impl(c, frames, n, S(stream));
}

fassmvs_status fassmvs_set_graph(fassmvs_ctx* c, int on)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    c->graph = on != 0;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_set_tuning(fassmvs_ctx* c, const fassmvs_tuning* t)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!t) return fail(c, FASSMVS_EINVAL, "tuning is NULL");
    FM_TRY(check_tuning(c, *t));
    c->tune = *t;
    c->tuned.clear();
    return FASSMVS_OK;
}

fassmvs_status fassmvs_autotune(fassmvs_ctx* c, const fassmvs_frame* frames, int n, void* stream,
                                fassmvs_tuning* chosen)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (n < 1 || n > 64 || !frames) return fail(c, FASSMVS_EINVAL, "1..64 frames");
    for (int f = 0; f < n; ++f) FM_TRY(check_frame(c, frames[f], c->cfg.levels, f));
    FM_TRY(set_device(c));
    cudaStream_t st = S(stream);
    // candidates: plane chunks of the persistent cost kernel x resident CTAs
    // x the aggregation's form (two-pass, or partial sums of concurrent
    // directions)
    std::vector<fassmvs_tuning> cand;
    for (int parts : {kSgmTwoPass, 2, 4, 8}) {
        if (parts > c->cfg.paths) continue;
        for (int chunk : {0, 64}) cand.push_back({chunk, 2, parts});
    }
    cand.push_back({0, 1, 0});
    cand.push_back({0, 0, 0});
    cudaEvent_t e0, e1;
    FM_TRY(cuda_check(c, cudaEventCreate(&e0), "event"));
    FM_TRY(cuda_check(c, cudaEventCreate(&e1), "event"));
    const bool prof = c->prof;
    c->prof = false;
    float best = 1e30f;
    fassmvs_tuning bt = c->tune;
    Stage sg;
    fassmvs_status rs = FASSMVS_OK;
    for (size_t i = 0; i <= cand.size() && rs == FASSMVS_OK; ++i) {
        // the first pass (the current setting) allocates scratch and warms up
        const fassmvs_tuning t = i == 0 ? c->tune : cand[i - 1];
        if ((rs = stage_prepare(c, frames, n, t.chunk_planes, &sg)) != FASSMVS_OK) break;
        cudaEventRecord(e0, st);
        rs = run_batch(c, frames, n, st, t, sg, nullptr);
        cudaEventRecord(e1, st);
        if (rs != FASSMVS_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) { rs = cuda_check(c, cudaGetLastError(), "autotune"); break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (i > 0 && ms < best) { best = ms; bt = t; }
    }
    c->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != FASSMVS_OK) return rs;
    const uint64_t shape = batch_signature(c, frames, n, nullptr);
    c->tuned[shape] = bt;
    if (chosen) *chosen = bt;
    if (const char* path = getenv("FASSMVS_TUNE_FILE")) {
        if (FILE* fp = fopen(path, "a")) {
            fprintf(fp, "{\"frames\": %d, \"shape\": \"%016llx\", \"chunk_planes\": %d, \"ctas_per_sm\": %d, "
                        "\"sgm_parts\": %d, \"ms\": %.3f}\n",
                    n, (unsigned long long)shape, bt.chunk_planes, bt.ctas_per_sm, bt.sgm_parts, best);
            fclose(fp);
        }
    }
    return FASSMVS_OK;
}

fassmvs_status fassmvs_estimate(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch,
                                const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* pl, float* depth,
                                float* normal, float* conf, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!c->cams) return fail(c, FASSMVS_EINVAL, "fassmvs_set_cameras was not called");
    if (!pl) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (n_nb != c->V) return fail(c, FASSMVS_EINVAL, "n_nb %d differs from the %d cameras set", n_nb, c->V);
    fassmvs_frame f;
    f.ref = ref; f.nbrs = nbrs; f.W = W; f.H = H; f.pitch = pitch; f.n_nb = n_nb;
    f.K = c->K; f.R = c->R.data(); f.t = c->t.data(); f.side = c->side.data();
    f.planes = *pl;
    f.depth = depth; f.normal = normal; f.conf = conf;
    return estimate_batch_impl(c, &f, 1, S(stream));
}

namespace {
// Enqueues one host-buffer estimate (fassmvs_estimate_host_async); *slot
// receives the device slot it used.
fassmvs_status estimate_host_enqueue(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch,
                                     const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* pl, float* depth,
                                     float* normal, float* conf, void* stream, int* slot)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!ref || !nbrs || !pl || !depth || !normal || !conf) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (W < 2 || H < 2 || pitch < W) return fail(c, FASSMVS_EINVAL, "image %dx%d with pitch %d", W, H, pitch);
    if (n_nb != c->V) return fail(c, FASSMVS_EINVAL, "n_nb %d differs from the %d cameras set", n_nb, c->V);
    if (n_nb > fm::kMaxViews) return fail(c, FASSMVS_EINVAL, "at most %d neighbours", fm::kMaxViews);
    for (int k = 0; k < n_nb; ++k)
        if (!nbrs[k]) return fail(c, FASSMVS_EINVAL, "neighbour %d is NULL", k);
    FM_TRY(set_device(c));
    cudaStream_t st = S(stream);
    if (!c->hp_h2d) {
        FM_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->hp_h2d, cudaStreamNonBlocking), "copy stream"));
        FM_TRY(cuda_check(c, cudaStreamCreateWithFlags(&c->hp_d2h, cudaStreamNonBlocking), "copy stream"));
        for (int i = 0; i < 2; ++i) {
            FM_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->hp_in[i], cudaEventDisableTiming), "event"));
            FM_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->hp_comp[i], cudaEventDisableTiming), "event"));
            FM_TRY(cuda_check(c, cudaEventCreateWithFlags(&c->hp_out[i], cudaEventDisableTiming), "event"));
        }
    }
    // per slot: the images with rows padded to 16 bytes (the cost kernel's
    // TMA staging of level 0 needs 16-byte aligned rows), then the maps
    const size_t dp = ((size_t)W + 15) & ~(size_t)15, img = dp * (size_t)H, npix = (size_t)W * H;
    const size_t img_bytes = (img * (size_t)(1 + n_nb) + 255) & ~(size_t)255;
    const size_t slot_bytes = img_bytes + sizeof(float) * npix * 5;
    if (slot_bytes != c->hp_slot_bytes) {
        // a new layout of the slots: every earlier call has finished with them
        for (int i = 0; i < 2; ++i)
            FM_TRY(cuda_check(c, cudaEventSynchronize(c->hp_out[i]), "earlier host estimate"));
        c->hp_slot_bytes = slot_bytes;
        c->hp_slot = 0;
    }
    void* base = nullptr;
    FM_TRY(ensure(c, "host_slots", 2 * slot_bytes, &base));
    const int s = c->hp_slot;
    unsigned char* sb = static_cast<unsigned char*>(base) + (size_t)s * slot_bytes;
    uint8_t* dimg = sb;
    float* dd = reinterpret_cast<float*>(sb + img_bytes);
    float* dnrm = dd + npix;
    float* dc = dnrm + 3 * npix;
    const uint8_t* dn[fm::kMaxViews];
    // images: once the estimate of this slot's previous use has read them
    FM_TRY(cuda_check(c, cudaStreamWaitEvent(c->hp_h2d, c->hp_comp[s], 0), "wait"));
    FM_TRY(cuda_check(c, cudaMemcpy2DAsync(dimg, dp, ref, (size_t)pitch, (size_t)W, (size_t)H,
                                           cudaMemcpyHostToDevice, c->hp_h2d), "host to device copy"));
    for (int k = 0; k < n_nb; ++k) {
        uint8_t* d = dimg + img * (size_t)(1 + k);
        FM_TRY(cuda_check(c, cudaMemcpy2DAsync(d, dp, nbrs[k], (size_t)pitch, (size_t)W, (size_t)H,
                                               cudaMemcpyHostToDevice, c->hp_h2d), "host to device copy"));
        dn[k] = d;
    }
    FM_TRY(cuda_check(c, cudaEventRecord(c->hp_in[s], c->hp_h2d), "event"));
    // the estimate: once the images are in and the previous use's maps are out
    FM_TRY(cuda_check(c, cudaStreamWaitEvent(st, c->hp_in[s], 0), "wait"));
    FM_TRY(cuda_check(c, cudaStreamWaitEvent(st, c->hp_out[s], 0), "wait"));
    FM_TRY(fassmvs_estimate(c, dimg, W, H, (int)dp, dn, n_nb, pl, dd, dnrm, dc, stream));
    FM_TRY(cuda_check(c, cudaEventRecord(c->hp_comp[s], st), "event"));
    // the maps
    FM_TRY(cuda_check(c, cudaStreamWaitEvent(c->hp_d2h, c->hp_comp[s], 0), "wait"));
    FM_TRY(cuda_check(c, cudaMemcpyAsync(depth, dd, sizeof(float) * npix, cudaMemcpyDeviceToHost, c->hp_d2h),
                      "device to host copy"));
    FM_TRY(cuda_check(c, cudaMemcpyAsync(normal, dnrm, sizeof(float) * 3 * npix, cudaMemcpyDeviceToHost,
                                         c->hp_d2h), "device to host copy"));
    FM_TRY(cuda_check(c, cudaMemcpyAsync(conf, dc, sizeof(float) * npix, cudaMemcpyDeviceToHost, c->hp_d2h),
                      "device to host copy"));
    FM_TRY(cuda_check(c, cudaEventRecord(c->hp_out[s], c->hp_d2h), "event"));
    c->hp_slot = s ^ 1;
    *slot = s;
    // the host images have been read
    return cuda_check(c, cudaEventSynchronize(c->hp_in[s]), "host to device copy");
}
}  // namespace

fassmvs_status fassmvs_estimate_host_async(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch,
                                           const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* pl,
                                           float* depth, float* normal, float* conf, void* stream)
{
    int slot = 0;
    return estimate_host_enqueue(c, ref, W, H, pitch, nbrs, n_nb, pl, depth, normal, conf, stream, &slot);
}

fassmvs_status fassmvs_estimate_host(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch,
                                     const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* pl, float* depth,
                                     float* normal, float* conf, void* stream)
{
    int slot = 0;
    FM_TRY(estimate_host_enqueue(c, ref, W, H, pitch, nbrs, n_nb, pl, depth, normal, conf, stream, &slot));
    // the maps copies run in order on one stream: this call's are the last
    return cuda_check(c, cudaEventSynchronize(c->hp_out[slot]), "device to host copy");
}

fassmvs_status fassmvs_profile_enable(fassmvs_ctx* c, int on)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    c->prof = on != 0;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_profile_read(fassmvs_ctx* c, double* ms, uint64_t* counts, int reset)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    FM_TRY(set_device(c));
    for (auto& r : c->pending) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
        if (e != cudaSuccess) {
            c->pending.clear();
            return cuda_check(c, e, "stage timer");
        }
        c->ms[r.stage] += t;
        c->cnt[r.stage] += 1;
    }
    c->pending.clear();
    for (int i = 0; i < FASSMVS_NSTAGES; ++i) {
        if (ms) ms[i] = c->ms[i];
        if (counts) counts[i] = c->cnt[i];
        if (reset) { c->ms[i] = 0.0; c->cnt[i] = 0; }
    }
    return FASSMVS_OK;
}

fassmvs_status fassmvs_sync(fassmvs_ctx* c)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    FM_TRY(set_device(c));
    cudaError_t e = c->last ? cudaStreamSynchronize(c->last) : cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    FM_TRY(cuda_check(c, e, "device error"));
    // deferred device-side flags: a connected-component walk that hit its cap;
    // a staged copy of the cost kernel that missed its bound (the kernel then
    // read global memory, so the volume is still right); a wait between rows
    // of the two-pass aggregation that gave up
    struct Flag {
        const char* buf;
        fassmvs_status status;
        const char* msg;
    };
    const Flag flags[3] = {
        {"ccl_err", FASSMVS_EINTERNAL, "a connected-component walk reached its bound (DoG filter)"},
        {"cost_err", FASSMVS_ETIMEOUT,
         "a staged copy of the cost kernel did not complete within its bound (the volume was read from global "
         "memory)"},
        {"sgm_err", FASSMVS_ETIMEOUT,
         "a row of the two-pass aggregation waited past its bound on a neighbouring row (the depth maps of that "
         "estimate are not valid)"}};
    // the checked build's bounds checks (always 0 in the default build)
    const unsigned sites[4] = {fm::check_take_cost(), fm::check_take_sgm(), fm::check_take_wave(),
                               fm::check_take_stages()};
    for (unsigned site : sites)
        if (site) return fail(c, FASSMVS_EINTERNAL, "bounds check failed at site 0x%x (checked build)", site);
    for (const Flag& fl : flags) {
        auto it = c->bufs.find(fl.buf);
        if (it == c->bufs.end() || !it->second.p) continue;
        int flag = 0;
        FM_TRY(cuda_check(c, cudaMemcpy(&flag, it->second.p, sizeof flag, cudaMemcpyDeviceToHost), "flag read"));
        if (flag) {
            cudaMemset(it->second.p, 0, sizeof flag);
            return fail(c, fl.status, "%s", fl.msg);
        }
    }
    return FASSMVS_OK;
}


// ---------------------------------------------------------------- plane selection
// Sec. 2.2.2 and Alg. 2: host-side FP64 geometry, no device work.  Planes are
// n^T X + delta = 0 in the reference frame; the ray X = s K^-1 (u, v, 1)^T
// meets the plane delta at s = -delta / (n^T r).

namespace {
struct V3 {
    double x, y, z;
};
V3 v3(double x, double y, double z) { return V3{x, y, z}; }
V3 mul(V3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
double vlen(V3 a) { return std::sqrt(dot(a, a)); }
V3 mat_vec(const double M[9], V3 a)
{
    return v3(M[0] * a.x + M[1] * a.y + M[2] * a.z, M[3] * a.x + M[4] * a.y + M[5] * a.z,
              M[6] * a.x + M[7] * a.y + M[8] * a.z);
}
// homogeneous image K (R X + t)
V3 image_h(const double K[9], const double R[9], const double t[3], V3 X)
{
    const V3 Y = mat_vec(R, X);
    return mat_vec(K, v3(Y.x + t[0], Y.y + t[1], Y.z + t[2]));
}
// sine of the angle between two rays (directions)
double sin_between(V3 a, V3 b) { return vlen(cross(a, b)) / (vlen(a) * vlen(b)); }
V3 corner_ray(const double Ki[9], int W, int H, int c)
{
    return mat_vec(Ki, v3((c & 1) ? W - 1 : 0, (c & 2) ? H - 1 : 0, 1.0));
}
}  // namespace

fassmvs_status fassmvs_debug_capture(fassmvs_ctx* c, int level)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (level < -1 || level >= c->cfg.levels) return fail(c, FASSMVS_EINVAL, "level -1 (off) or 0..levels-1");
    c->dbg_level = level;
    memset(c->dbg_dims, 0, sizeof c->dbg_dims);
    return FASSMVS_OK;
}

fassmvs_status fassmvs_debug_capture_warp(fassmvs_ctx* c, int plane, int view)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (plane < -1 || view < -1 || view >= fm::kMaxViews || (plane < 0) != (view < 0))
        return fail(c, FASSMVS_EINVAL, "plane and view both -1 (off) or both >= 0");
    c->dbg_warp_g = plane;
    c->dbg_warp_k = view;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_debug_dump(fassmvs_ctx* c, int level, int what, void* dst, size_t cap, size_t* bytes,
                                  int32_t dims[5])
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (level != c->dbg_level || c->dbg_dims[0] == 0)
        return fail(c, FASSMVS_EINVAL, "level %d was not captured by the last estimate", level);
    static const char* const names[9] = {"dbg:S",    "dbg:lo",   "dbg:dI",   "dbg:agg", "dbg:gwin",
                                         "dbg:draw", "dbg:dmed", "dbg:nrm", "dbg:warp"};
    if (what < 0 || what > 8) return fail(c, FASSMVS_EINVAL, "what 0..8");
    const size_t np = (size_t)c->dbg_dims[0] * c->dbg_dims[1], nv = np * c->dbg_dims[3];
    const size_t need[9] = {2 * nv, 4 * np, 8 * np, 2 * nv, 4 * np, 4 * np, 4 * np, 12 * np, 4 * np};
    if (bytes) *bytes = need[what];
    if (dims) memcpy(dims, c->dbg_dims, sizeof c->dbg_dims);
    if (!dst) return FASSMVS_OK;
    if (cap < need[what]) return fail(c, FASSMVS_EINVAL, "%zu bytes needed", need[what]);
    auto it = c->bufs.find(names[what]);
    if (it == c->bufs.end() || !it->second.p) return fail(c, FASSMVS_EINVAL, "nothing captured");
    FM_TRY(set_device(c));
    FM_TRY(cuda_check(c, cudaStreamSynchronize(c->last), "sync"));
    return cuda_check(c, cudaMemcpy(dst, it->second.p, need[what], cudaMemcpyDefault), "dump copy");
}

fassmvs_status fassmvs_debug_inject(fassmvs_ctx* c, int mode)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (mode != 0 && mode != 1) return fail(c, FASSMVS_EINVAL, "mode 0 (off) or 1 (staging waits give up)");
    c->inject = mode;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_plane_bounds(const double K[9], int W, int H, const double n[3], double d_min, double d_max,
                                    double* delta_min, double* delta_max)
{
    if (!K || !n || !delta_min || !delta_max) return fail(nullptr, FASSMVS_EINVAL, "NULL argument");
    double Ki[9];
    if (!k_inverse(K, Ki) || W < 1 || H < 1) return fail(nullptr, FASSMVS_EINVAL, "bad K or image size");
    if (!(d_min > 0.0) || !(d_max > d_min)) return fail(nullptr, FASSMVS_EINVAL, "need 0 < d_min < d_max");
    const V3 nn = v3(n[0], n[1], n[2]);
    if (!(std::fabs(vlen(nn) - 1.0) < 1e-9)) return fail(nullptr, FASSMVS_EINVAL, "n must be a unit vector");
    double lo = HUGE_VAL, hi = 0.0;
    for (int c = 0; c < 4; ++c) {
        const V3 r = corner_ray(Ki, W, H, c);
        if (!(dot(nn, r) < 0.0)) return fail(nullptr, FASSMVS_EINVAL, "a corner ray does not meet the planes");
        lo = std::min(lo, std::fabs(dot(nn, mul(r, d_min))));
        hi = std::max(hi, std::fabs(dot(nn, mul(r, d_max))));
    }
    *delta_min = lo;
    *delta_max = hi;
    return FASSMVS_OK;
}

fassmvs_status fassmvs_cross_ratio_planes(const double K[9], int W, int H, int n_cams, const double* R,
                                          const double* t, const double n[3], double delta_min, double delta_max,
                                          int max_planes, double* deltas, int* count, int* camera,
                                          fassmvs_planes* uniform)
{
    if (!K || !R || !t || !n || !count) return fail(nullptr, FASSMVS_EINVAL, "NULL argument");
    double Ki[9];
    if (!k_inverse(K, Ki) || W < 1 || H < 1) return fail(nullptr, FASSMVS_EINVAL, "bad K or image size");
    if (n_cams < 1) return fail(nullptr, FASSMVS_EINVAL, "need at least one camera");
    if (!(delta_min > 0.0) || !(delta_max > delta_min))
        return fail(nullptr, FASSMVS_EINVAL, "need 0 < delta_min < delta_max");
    if (deltas && max_planes < 2) return fail(nullptr, FASSMVS_EINVAL, "max_planes must be >= 2");
    const V3 nn = v3(n[0], n[1], n[2]);
    if (!(std::fabs(vlen(nn) - 1.0) < 1e-9)) return fail(nullptr, FASSMVS_EINVAL, "n must be a unit vector");
    for (int i = 0; i < n_cams; ++i) {
        const double* Ri = R + 9 * i;
        const double* ti = t + 3 * i;
        // C_i = -R_i^T t_i must lie in front of Pi_min
        const V3 Ci = v3(-(Ri[0] * ti[0] + Ri[3] * ti[1] + Ri[6] * ti[2]), -(Ri[1] * ti[0] + Ri[4] * ti[1] + Ri[7] * ti[2]),
                         -(Ri[2] * ti[0] + Ri[5] * ti[1] + Ri[8] * ti[2]));
        if (!(dot(nn, Ci) + delta_min > 0.0))
            return fail(nullptr, FASSMVS_EINVAL, "camera %d is not in front of the nearest plane", i);
    }
    // p_ref and camera k: the longest image segment between the bounding planes
    int k = -1, corner = 0;
    double L = 0.0;
    for (int i = 0; i < n_cams; ++i)
        for (int c = 0; c < 4; ++c) {
            const V3 r = corner_ray(Ki, W, H, c);
            const double nr = dot(nn, r);
            if (!(nr < 0.0)) return fail(nullptr, FASSMVS_EINVAL, "a corner ray does not meet the planes");
            const V3 a = image_h(K, R + 9 * i, t + 3 * i, mul(r, -delta_min / nr));
            const V3 b = image_h(K, R + 9 * i, t + 3 * i, mul(r, -delta_max / nr));
            if (!(a.z > 0.0 && b.z > 0.0)) continue;
            const double len = std::hypot(a.x / a.z - b.x / b.z, a.y / a.z - b.y / b.z);
            if (len > L) {
                L = len;
                k = i;
                corner = c;
            }
        }
    if (k < 0) return fail(nullptr, FASSMVS_EINVAL, "no corner segment between the planes in any camera");
    const double* Rk = R + 9 * k;
    const double* tk = t + 3 * k;
    const V3 V = corner_ray(Ki, W, H, corner);
    const double nV = dot(nn, V);
    const V3 xmin = image_h(K, Rk, tk, mul(V, -delta_min / nV));
    const V3 xmax = image_h(K, Rk, tk, mul(V, -delta_max / nV));
    const double pmin[2] = {xmin.x / xmin.z, xmin.y / xmin.z}, pmax[2] = {xmax.x / xmax.z, xmax.y / xmax.z};
    const double kx = (pmin[0] - pmax[0]) / L, ky = (pmin[1] - pmax[1]) / L;
    // rays of camera k; the epipole's ray runs from C_k towards C_ref, whose
    // homogeneous image is K t_k: its direction is t_k whatever side C_ref is on
    const V3 Ve = v3(tk[0], tk[1], tk[2]);
    const V3 Vmin = mat_vec(Ki, v3(pmin[0], pmin[1], 1.0)), Vmax = mat_vec(Ki, v3(pmax[0], pmax[1], 1.0));
    const double s_mm = sin_between(Vmin, Vmax), s_emax = sin_between(Ve, Vmax);
    // distance of the plane whose image of p_ref is `a` pixels from p_max
    auto delta_at = [&](double a) {
        const V3 Vi = mat_vec(Ki, v3(pmax[0] + a * kx, pmax[1] + a * ky, 1.0));
        const double Q = sin_between(Ve, Vi) * s_mm / (s_emax * sin_between(Vmin, Vi));
        return Q * delta_max * delta_min / (Q * delta_max - (delta_max - delta_min));
    };
    const int steps = (int)std::ceil(L);
    *count = steps + 1;
    if (camera) *camera = k;
    if (deltas && steps + 1 > max_planes)
        return fail(nullptr, FASSMVS_EINVAL, "%d planes needed, more than max_planes", steps + 1);
    if (deltas) {
        for (int i = 0; i < steps; ++i) deltas[i] = delta_at(i);
        deltas[steps] = delta_min;
    }
    if (uniform) {
        // uniform in inverse distance, covering [delta_min, delta_max]: what
        // the estimate sweeps.  The image of p_ref moves along the epipolar
        // line as a projective function of 1/delta, so its speed is monotone
        // and largest at one end; the step is the smaller of the one-pixel
        // steps at the two ends, and then no step moves p_ref by more than a
        // pixel.  The range is then split evenly so that the last plane is
        // Pi_min itself (past it p_ref would move faster still).  A segment
        // shorter than a pixel gives the two bounding planes.
        const double range = 1.0 / delta_min - 1.0 / delta_max;
        double inv_step = range;
        if (L > 1.0) {
            inv_step = std::min(1.0 / delta_at(1.0) - 1.0 / delta_max, 1.0 / delta_min - 1.0 / delta_at(L - 1.0));
        }
        const int32_t G0 = (int32_t)std::ceil(range / inv_step - 1e-9) + 1;
        uniform->n[0] = n[0];
        uniform->n[1] = n[1];
        uniform->n[2] = n[2];
        uniform->rho_far = 1.0 / delta_max;
        uniform->drho = range / (G0 - 1);
        uniform->G0 = G0;
    }
    return FASSMVS_OK;
}

fassmvs_status fassmvs_dog_filter(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch, float* depth,
                                  float* normal, float* conf, uint8_t* mask, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!ref || W < 1 || H < 1 || pitch < W) return fail(c, FASSMVS_EINVAL, "bad reference image");
    if ((depth || normal || conf) && !(depth && normal && conf))
        return fail(c, FASSMVS_EINVAL, "depth, normal and conf go together");
    if ((size_t)W * H >= ((size_t)1 << 31)) return fail(c, FASSMVS_EINVAL, "image too large");
    FM_TRY(set_device(c));
    cudaStream_t st = S(stream);
    c->last = st;
    const size_t np = (size_t)W * H;
    void *m, *tmp, *parent, *size, *err;
    if (mask) m = mask;
    else FM_TRY(ensure(c, "dog_mask", np, &m));
    FM_TRY(ensure(c, "dog_tmp", np, &tmp));
    FM_TRY(ensure(c, "ccl_parent", np * sizeof(int), &parent));
    FM_TRY(ensure(c, "ccl_size", np * sizeof(int), &size));
    const bool fresh = !c->bufs.count("ccl_err");
    FM_TRY(ensure(c, "ccl_err", sizeof(int), &err));
    if (fresh) FM_TRY(cuda_check(c, cudaMemsetAsync(err, 0, sizeof(int), st), "memset"));
    fm::launch_dog_mask(ref, W, H, pitch, dog_weights(), (uint8_t*)m, (uint8_t*)tmp, (int*)parent, (int*)size,
                        (int*)err, st);
    if (depth) fm::launch_apply_mask((const uint8_t*)m, W, H, depth, normal, conf, st);
    return launch_status(c, "dog filter launch");
}

fassmvs_status fassmvs_geo_filter(fassmvs_ctx* c, float* depth, float* normal, float* conf, int W, int H,
                                  const double K[9], int n, const float* const* depths, const double* R,
                                  const double* t, double eta_r, int eta_h, uint8_t* hits, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!depth || !K || (n > 0 && (!depths || !R || !t))) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (W < 1 || H < 1 || n < 0 || n > fm::kMaxViews) return fail(c, FASSMVS_EINVAL, "bad size or map count");
    if (!(eta_r > 0.0) || eta_h < 0) return fail(c, FASSMVS_EINVAL, "eta_r must be > 0, eta_h >= 0");
    if (K[1] != 0.0 || K[3] != 0.0 || K[6] != 0.0 || K[7] != 0.0 || K[8] != 1.0 || K[0] == 0.0 || K[4] == 0.0)
        return fail(c, FASSMVS_EINVAL, "K must be [[fx 0 cx][0 fy cy][0 0 1]]");
    fm::GeoArgs g;
    memset(&g, 0, sizeof g);
    g.W = W; g.H = H; g.n = n; g.eta_h = eta_h; g.eta_r = eta_r;
    g.fx = K[0]; g.fy = K[4]; g.cx = K[2]; g.cy = K[5];
    for (int k = 0; k < n; ++k) {
        if (!depths[k]) return fail(c, FASSMVS_EINVAL, "depth map %d is NULL", k);
        if (depths[k] == depth) return fail(c, FASSMVS_EINVAL, "depth map %d is the filtered map", k);
        g.dk[k] = depths[k];
        for (int i = 0; i < 9; ++i) g.R[k][i] = R[9 * k + i];
        for (int i = 0; i < 3; ++i) g.t[k][i] = t[3 * k + i];
    }
    FM_TRY(set_device(c));
    cudaStream_t st = S(stream);
    c->last = st;
    fm::launch_geo_filter(g, depth, normal, conf, hits, st);
    return launch_status(c, "geometric filter launch");
}

const char* fassmvs_last_error(const fassmvs_ctx* c)
{
    if (c) return c->err.c_str();
    return t_err.c_str();
}

uint64_t fassmvs_launch_count(const fassmvs_ctx* c)
{
    (void)c;
    return fm::launches();
}

}  // extern "C"
