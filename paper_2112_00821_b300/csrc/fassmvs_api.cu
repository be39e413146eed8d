// C-ABI layer of the B300 FaSS-MVS library: argument validation, the host-side
// FP64 camera algebra (rank-1 homography factors), scratch management within
// the context's memory budget, and the coarse-to-fine level loop of Sec. 2.1.
// Every compute step runs in the kernels of cost.cu, sgm.cu and stages.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>
#include <atomic>

#include "../../include/fassmvs.h"
#include "fm_internal.cuh"

namespace fm {
static std::atomic<uint64_t> g_launches{0};
uint64_t launches() { return g_launches.load(); }
void count_launch(int n) { g_launches.fetch_add((uint64_t)n); }
}  // namespace fm

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
    struct Rec { cudaEvent_t a, b; int stage; };
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> pending;
    double ms[FASSMVS_NSTAGES] = {};
    uint64_t cnt[FASSMVS_NSTAGES] = {};
};

namespace {

thread_local std::string t_err;

fassmvs_status fail(fassmvs_ctx* c, fassmvs_status s, const char* fmt, ...)
    __attribute__((format(printf, 3, 4)));

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

}  // namespace

void fm::set_error(const char* msg) { t_err = msg; }

namespace {

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

// Brackets the launches of one stage with events when profiling is on.
struct StageTimer {
    fassmvs_ctx* c;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageTimer(fassmvs_ctx* c_, int s, cudaStream_t st_) : c(c_), stage(s), st(st_)
    {
        if (c && c->prof && (a = take_event(c))) cudaEventRecord(a, st);
    }
    ~StageTimer()
    {
        if (!a) return;
        cudaEvent_t b = take_event(c);
        if (!b) { c->pool.push_back(a); return; }
        cudaEventRecord(b, st);
        c->pending.push_back({a, b, stage});
    }
};

fassmvs_status set_device(fassmvs_ctx* c) { return cuda_check(c, cudaSetDevice(c->device), "cudaSetDevice"); }

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

}  // namespace

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
    return sgm_impl(c, Sv, lo, dI, img, W, W, H, D, Ds, prm, fm::kCensusMax * fm::kMaxViews, Sbar, S(stream));
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
    fm::launch_wta_refine(Sbar, lo, W, H, D, Ds, (const float*)delta, intr(K), nf, depth, gwin, S(stream));
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
                           const double K[9], double drho, int dmax, int8_t* dI, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!dc || !nc || !dI || !K || Wc < 1 || Hc < 1 || W < 1 || H < 1 || dmax < 0 || dmax > 127)
        return fail(c, FASSMVS_EINVAL, "bad dsn arguments");
    FM_TRY(set_device(c));
    fm::launch_dsn(dc, nc, Wc, Hc, W, H, intr(K), (float)drho, dmax, dI, S(stream));
    c->last = S(stream);
    return launch_status(c, "dsn launch");
}

fassmvs_status fassmvs_estimate(fassmvs_ctx* c, const uint8_t* ref, int W, int H, int pitch,
                                const uint8_t* const* nbrs, int n_nb, const fassmvs_planes* pl, float* depth,
                                float* normal, float* conf, void* stream)
{
    if (!c) return fail(nullptr, FASSMVS_EINVAL, "ctx is NULL");
    if (!c->cams) return fail(c, FASSMVS_EINVAL, "fassmvs_set_cameras was not called");
    if (!ref || !nbrs || !pl || !depth || !normal || !conf) return fail(c, FASSMVS_EINVAL, "NULL argument");
    if (n_nb != c->V) return fail(c, FASSMVS_EINVAL, "n_nb %d differs from the %d cameras set", n_nb, c->V);
    if (W < 2 || H < 2 || pitch < W) return fail(c, FASSMVS_EINVAL, "bad image size or pitch");
    const fassmvs_config& cfg = c->cfg;
    const int L = cfg.levels;
    if (((W - 1) >> (L - 1)) + 1 < 2 || ((H - 1) >> (L - 1)) + 1 < 2)
        return fail(c, FASSMVS_EINVAL, "image too small for %d levels", L);
    if (pl->G0 < 1) return fail(c, FASSMVS_EINVAL, "G0 must be >= 1");
    const int Gtop = (pl->G0 - 1) / (1 << (L - 1)) + 1;
    if (Gtop > fm::kMaxSlots) return fail(c, FASSMVS_EINVAL, "top level has %d planes (> 256, Sec. 3.2 cap)", Gtop);
    FM_TRY(set_device(c));
    cudaStream_t st = S(stream);
    c->last = st;
    const int V = c->V;
    int nL = 0, nR = 0;
    for (int k = 0; k < V; ++k) { if (c->side[k] < 0) ++nL; else ++nR; }
    const int nmax = nL > nR ? nL : nR;
    const int P1 = cfg.p1 * nmax;
    uint16_t lut[256];
    p2_table(P1, cfg.alpha, cfg.beta, lut);
    fassmvs_sgm_params prm{cfg.paths, cfg.variant, P1, cfg.p2 * nmax, cfg.dmax, cfg.adaptive_p2 ? lut : nullptr};

    // image pyramids (level 0 is the caller's)
    int Ws[8], Hs[8], Ps[8];
    const uint8_t* img[8][fm::kMaxViews + 1];
    Ws[0] = W; Hs[0] = H; Ps[0] = pitch;
    img[0][0] = ref;
    for (int k = 0; k < V; ++k) img[0][k + 1] = nbrs[k];
    StageTimer* tpyr = new StageTimer(c, FASSMVS_STAGE_PYRAMID, st);
    for (int l = 1; l < L; ++l) {
        Ws[l] = (Ws[l - 1] + 1) / 2;
        Hs[l] = (Hs[l - 1] + 1) / 2;
        Ps[l] = Ws[l];
        void* p;
        char name[32];
        snprintf(name, sizeof name, "pyr%d", l);
        fassmvs_status es = ensure(c, name, (size_t)(V + 1) * Ws[l] * Hs[l], &p);
        if (es != FASSMVS_OK) { delete tpyr; return es; }
        for (int k = 0; k <= V; ++k) {
            uint8_t* o = (uint8_t*)p + (size_t)k * Ws[l] * Hs[l];
            fm::launch_pyramid_down(img[l - 1][k], Ws[l - 1], Hs[l - 1], Ps[l - 1], o, Ps[l], st);
            img[l][k] = o;
        }
    }
    delete tpyr;
    float* dprev = nullptr;
    float* nprev = nullptr;
    for (int l = L - 1; l >= 0; --l) {
        const int w = Ws[l], h = Hs[l];
        const size_t np = (size_t)w * h;
        const double sc = (double)(1 << l);
        const double Kl[9] = {c->K[0] / sc, c->K[1] / sc, c->K[2] / sc, 0.0, c->K[4] / sc, c->K[5] / sc, 0.0, 0.0, 1.0};
        const int Gl = (pl->G0 - 1) / (1 << l) + 1;
        const double drl = pl->drho * sc;
        const int D = (l == L - 1) ? Gl : (cfg.D[l] < Gl ? cfg.D[l] : Gl);
        const int Ds = (D + 7) & ~7;
        void *pS, *pSb, *pdraw, *pdmed, *pnraw, *pnrm, *plo = nullptr, *pdI = nullptr;
        FM_TRY(ensure(c, "S", sizeof(uint16_t) * np * Ds, &pS));
        FM_TRY(ensure(c, "Sbar", sizeof(uint16_t) * np * Ds, &pSb));
        FM_TRY(ensure(c, "draw", sizeof(float) * np, &pdraw));
        FM_TRY(ensure(c, "nraw", sizeof(float) * 3 * np, &pnraw));
        if (l > 0) {
            FM_TRY(ensure(c, (l & 1) ? "dmedA" : "dmedB", sizeof(float) * np, &pdmed));
            FM_TRY(ensure(c, (l & 1) ? "nrmA" : "nrmB", sizeof(float) * 3 * np, &pnrm));
        } else {
            pdmed = depth;
            pnrm = normal;
        }
        if (l < L - 1) {
            FM_TRY(ensure(c, "lo", sizeof(int32_t) * np, &plo));
            if (cfg.variant == 1) FM_TRY(ensure(c, "dI", 8 * np, &pdI));
            StageTimer tm(c, FASSMVS_STAGE_WINDOW, st);
            float nf[3] = {(float)pl->n[0], (float)pl->n[1], (float)pl->n[2]};
            fm::launch_window(dprev, Ws[l + 1], Hs[l + 1], w, h, intr(Kl), nf, (float)pl->rho_far, (float)drl, Gl, D,
                              (int32_t*)plo, st);
            if (cfg.variant == 1) {
                fm::launch_dsn(dprev, nprev, Ws[l + 1], Hs[l + 1], w, h, intr(Kl), (float)drl, cfg.dmax, (int8_t*)pdI, st);
            }
        } else if (cfg.variant == 1) {
            FM_TRY(ensure(c, "dI", 8 * np, &pdI));
            FM_TRY(cuda_check(c, cudaMemsetAsync(pdI, 0, 8 * np, st), "memset dI"));
        }
        FM_TRY(cost_volume_impl(c, img[l][0], &img[l][1], V, c->side.data(), w, h, Ps[l], Kl, c->R.data(),
                                c->t.data(), pl->n, pl->rho_far, drl, Gl, (const int32_t*)plo, D, Ds,
                                (uint16_t*)pS, st));
        FM_TRY(sgm_impl(c, (const uint16_t*)pS, (const int32_t*)plo, (const int8_t*)pdI, img[l][0], Ps[l], w, h, D, Ds,
                        &prm, fm::kCensusMax * nmax, (uint16_t*)pSb, st));
        void* delta;
        FM_TRY(ensure(c, "delta", sizeof(float) * (size_t)Gl, &delta));
        float nf[3] = {(float)pl->n[0], (float)pl->n[1], (float)pl->n[2]};
        {
            StageTimer tm(c, FASSMVS_STAGE_WTA, st);
            fm::launch_wta_refine((const uint16_t*)pSb, (const int32_t*)plo, w, h, D, Ds, (const float*)delta, intr(Kl),
                                  nf, cfg.median5 ? (float*)pdraw : (float*)pdmed, nullptr, st);
        }
        if (cfg.median5) {
            StageTimer tm(c, FASSMVS_STAGE_MEDIAN, st);
            fm::launch_median5((const float*)pdraw, w, h, (float*)pdmed, st);
        }
        StageTimer tmn(c, FASSMVS_STAGE_NORMALS, st);
        fm::launch_normals((const float*)pdmed, img[l][0], Ps[l], w, h, intr(Kl), cfg.normal_radius, cfg.normal_beta,
                           (float*)pnraw, (float*)pnrm, nf, cfg.rho_deg, l == 0 ? conf : nullptr, st);
        FM_TRY(launch_status(c, "level launch"));
        dprev = (float*)pdmed;
        nprev = (float*)pnrm;
    }
    return FASSMVS_OK;
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
    return cuda_check(c, e, "device error");
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
