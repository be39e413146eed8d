// Internal declarations shared by the kernels and the C-ABI layer of the
// B300 FaSS-MVS library.  Nothing here is part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fm {

// ---------------------------------------------------------------- checked build
// With -DFASSMVS_CHECKED (libfassmvs_checked.so) the kernels test the indices
// they form into shared and global memory before each access: FM_IN(i, n,
// site) is true for 0 <= i < n; otherwise it records `site` in the
// translation unit's check word (the first failure wins) and the access is
// skipped, so nothing outside a buffer is read or written and no kernel traps.
// fassmvs_sync turns a recorded site into FASSMVS_EINTERNAL.  Sites: 0x1nn
// cost.cu, 0x2nn sgm.cu, 0x3nn sgm_wave.cu, 0x4nn stages.cu.  In the default
// build every check is the constant true.
#if defined(FASSMVS_CHECKED) && defined(__CUDACC__)
static __device__ unsigned int fm_check_word;
__device__ __forceinline__ bool fm_in(long long i, long long n, unsigned site)
{
    if (i >= 0 && i < n) return true;
    atomicCAS(&fm_check_word, 0u, site);
    return false;
}
#define FM_IN(i, n, site) ::fm::fm_in((long long)(i), (long long)(n), (site))
// the translation unit's recorded site (0: none), cleared once read
#define FM_CHECK_TAKE(fn)                                                          \
    unsigned fn()                                                                  \
    {                                                                              \
        unsigned v = 0, z = 0;                                                     \
        cudaMemcpyFromSymbol(&v, fm_check_word, sizeof v);                         \
        if (v) cudaMemcpyToSymbol(fm_check_word, &z, sizeof z);                    \
        return v;                                                                  \
    }
#else
#define FM_IN(i, n, site) true
#define FM_CHECK_TAKE(fn) \
    unsigned fn() { return 0u; }
#endif
// per translation unit
unsigned check_take_cost();
unsigned check_take_sgm();
unsigned check_take_wave();
unsigned check_take_stages();

constexpr int kMaxViews = 16;     // neighbour views per reference frame
constexpr int kMaxSlots = 256;    // planes per pixel window (32 lanes x 8 slots)
constexpr int kCensusMax = 62;    // informative bits of a 9x7 census string

// ---------------------------------------------------------------- cameras
// Per view, the rank-1 form of the plane-induced homography
//   H(rho) = A - rho * e c^T,  A = K R K^-1, e = K t, c = K^-T n,
// (Eq. homography with rho = 1 / delta), precomputed on the host in FP64.
struct ViewGeom {
    double A[kMaxViews][9];
    double e[kMaxViews][3];
    double c[kMaxViews][3];
};

// One level of the sweep: G planes with 1/delta_g = rho0 + g * drho.
struct LevelPlanes {
    double rho0, drho;
    int G, V;
    double xc, yc;    // image centre, where the homographies are normalised
};

// Device tables built once per level by prep_level_kernel:
//   htab[(g * V + k) * 18 + i]     H_{g,k} entry i as (hi, lo) float pairs:
//                                   i in 0..8 -> hi, 9..17 -> lo (row-major)
//   delta[g]                        plane distance 1 / (rho0 + g drho)
void launch_prep_level(const ViewGeom& vg, const LevelPlanes& lp, float* htab, float* delta,
                       cudaStream_t st);

// ---------------------------------------------------------------- cost volume
struct ViewPtrs {
    const uint8_t* img[kMaxViews];
    int side[kMaxViews];          // -1 left, +1 right
};

struct CostArgs {
    int cost;                     // 0: census 9x7 Hamming, 1: NCC 5x5
    const uint64_t* cref;         // reference census [H][W] (census)
    const uint8_t* ref;           // reference image, rows ref_pitch bytes apart (NCC)
    int ref_pitch;
    ViewPtrs views;
    int V, W, H, pitch;
    int nL, nR, nmax;
    uint64_t mL, mR;              // ceil(2^32 / nL), ceil(2^32 / nR)
    const float* htab;
    const int32_t* lo;            // may be null (window starts at 0)
    int D, Ds, G;
    // voxel (pixel p, slot s) at S[p * pstride + (s >> bshift) * bstride +
    // (s & (2^bshift - 1))]: [H][W][Ds] is pstride = Ds, bshift = 3,
    // bstride = 8; the 16-plane-blocked [Ds / 16][H][W][16] (Ds a multiple of
    // 16) is pstride = 16, bshift = 4, bstride = 16 W H
    size_t pstride, bstride;
    int bshift;
    uint16_t* S;
    // staging of the neighbour images (may be null): V tensor maps (CUtensorMap,
    // 128 B each, 64-byte aligned, global memory) of the views' uint8 images
    // with a kStageBX x kStageBY box; and an error word raised when a staged
    // copy does not complete within its bound (the kernel then reads global
    // memory, so results are unchanged)
    const void* tmaps;
    int* err;
    // test hook: plan the staging boxes but issue no copies, with a wait
    // bound of about a millisecond, so that every staged wait gives up
    int stage_test;
    // debug capture (may be null): the warped values minus 128 of plane
    // dbg_g, view dbg_k at every pixel whose tile sampled that pair, float
    // [H][W], exactly as the census reads them
    float* dbg_warp;
    int dbg_g, dbg_k;
};
constexpr int kStageBX = 128, kStageBY = 80;
void launch_cost(const CostArgs& a, cudaStream_t st);
// multi-frame form: items[i] = (frame, tile x, tile y, chunk | chunks << 16);
// ctas > 0 persistent CTAs pulling items from *counter, else one CTA per item;
// ncc: every frame's args use the NCC cost (else the census); dbg: the kernel
// that copies a chosen pair's warped tile to dbg_warp (a separate
// instantiation, so the usual one holds none of that code)
void launch_cost_batch(const CostArgs* args, const int4* items, int n_items, int* counter, int ctas, bool ncc,
                       bool dbg, cudaStream_t st);
int cost_tiles_x(int W);
int cost_tiles_y(int H);

// ---------------------------------------------------------------- SGM
struct SgmArgs {
    const uint16_t* S;
    const int32_t* lo;
    const int8_t* dI;
    const uint8_t* img;
    int W, H, D, Ds, img_pitch;
    size_t pstride, bstride;      // volume layout, as in CostArgs
    int bshift;
    int paths, variant, p1, p2, dmax;
    int use_lut;
    uint16_t lut[256];
    uint16_t* Sbar;
    size_t part_stride;           // elements between partial sums (batch form)
};
void launch_sgm(const SgmArgs& a, cudaStream_t st);
// path lines of direction r for a W x H image, padded to whole CTAs
int sgm_lines(int W, int H, int r);
// multi-frame, multi-direction form: up to kSgmBatch frames and 8 direction
// slots per launch, passed by value.  Slot j runs direction r[j] (steps
// dx[j], dy[j]) into partial sum part[j] (at Sbar + part * part_stride of each
// frame), writing it when first[j], else adding to it.  seg[j][f] is the first
// path line of (slot j, frame f), padded to whole CTAs; seg[j][nframes] ==
// seg[j + 1][0] and seg[nslots - 1][nframes] is the total.
constexpr int kSgmBatch = 32;
// resident image pyramid of a reference frame and its views (serving form):
// img[l][0] the reference, img[l][k + 1] view k, rows pitch[l] bytes apart
// (level 0 too)
struct PyrSet {
    const uint8_t* img[8][kMaxViews + 1];
    int pitch[8];
};
struct SgmBatch {
    SgmArgs a[kSgmBatch];
    int nframes, nslots;
    int r[8], dx[8], dy[8], part[8], first[8];
    int seg[8][kSgmBatch + 1];
};
void sgm_dir_of(int r, int* dx, int* dy);
void launch_sgm_batch(const SgmBatch& b, cudaStream_t st);

// ---------------------------------------------------------------- per-pixel stages
void launch_pyramid_down(const uint8_t* in, int W, int H, int pitch_in, uint8_t* out,
                         int pitch_out, cudaStream_t st);
void launch_census(const uint8_t* img, int W, int H, int pitch, uint64_t* out, cudaStream_t st);

struct Intr {
    float fx, fy, cx, cy;
};

#ifdef __CUDACC__
// Sub-plane refinement of the winner (Sec. 2.3.4): the vertex of the parabola
// through the costs (cm, c0, cp) at the plane distances (xm, x0, xp), clamped
// to [min(xm, xp), max(xm, xp)]; x0 where the three are not convex.  Every
// operation rounds on its own (no contraction into fused multiply-adds), so
// every kernel that takes the winner gets the same bits.
__device__ __forceinline__ float wta_vertex(float x0, float xm, float xp, float c0, float cm, float cp)
{
    const float A = __fmul_rn(__fsub_rn(x0, xm), __fsub_rn(c0, cp));
    const float B = __fmul_rn(__fsub_rn(x0, xp), __fsub_rn(c0, cm));
    const float den = __fsub_rn(A, B);
    if (!(den > 0.0f)) return x0;
    const float num = __fsub_rn(__fmul_rn(__fsub_rn(x0, xm), A), __fmul_rn(__fsub_rn(x0, xp), B));
    const float xs = __fsub_rn(x0, __fdiv_rn(__fmul_rn(0.5f, num), den));
    return fminf(fmaxf(xs, fminf(xm, xp)), fmaxf(xm, xp));
}
// Depth at pixel (x, y) of the plane n^T X + xs = 0 (Sec. 2.2.1): -xs over
// n^T K^-1 (x, y, 1)^T, each operation rounded on its own.
__device__ __forceinline__ float wta_depth(float xs, int x, int y, Intr K, float n0, float n1, float n2)
{
    const float u = __fdiv_rn(__fsub_rn((float)x, K.cx), K.fx);
    const float v = __fdiv_rn(__fsub_rn((float)y, K.cy), K.fy);
    const float ray = __fadd_rn(__fadd_rn(__fmul_rn(n0, u), __fmul_rn(n1, v)), n2);
    return __fdiv_rn(-xs, ray);
}
#endif

// ---------------------------------------------------------------- two-pass SGM
// The aggregation and the winner-takes-all in two wavefront passes (sgm_wave.cu):
// pass A runs the four paths that come from the left and from the row above,
// top row first, and writes the sum of its paths (T1, the cost volume's
// layout); pass B runs the other four from the bottom-right corner, adds T1 and
// takes the winner, the parabola and the depth in place (and, for a debug
// capture, writes the whole aggregate to Sbar).  A block of kWaveRows image rows
// is one CTA, one warp per row; the previous row's path costs reach the next
// warp through shared memory and the next block through a ring in global
// memory (kWaveRing columns per block boundary, or a whole row).
constexpr int kWaveRows = 4;
constexpr int kWaveRing = 32;
constexpr int kWaveBatch = 16;
struct WaveFrame {
    SgmArgs a;                    // S, lo, dI, img, sizes, layout, penalties (a.Sbar: debug aggregate or null)
    uint16_t* T1;                 // pass A sums, the cost volume's layout
    const float* delta;           // plane distances (winner-takes-all)
    int G;                        // planes of the level list (entries of delta)
    Intr K;
    float n0, n1, n2;
    float* depth;
    int32_t* gwin;                // winning plane per pixel (may be null)
    uint4* gring;                 // per block boundary: [ring][3][32] path costs
    int4* gscal;                  // per block boundary: [ring][4] scalars
    int ring;                     // columns of each ring (a power of two)
    int* gflag;                   // per block boundary: producer columns done, consumer columns done
    int nblocks;                  // ceil(H / kWaveRows)
};
struct WaveBatch {
    WaveFrame f[kWaveBatch];
    int nframes;
    int item0[kWaveBatch + 1];    // first CTA item of each frame (items in frame order)
    int* ticket;                  // item counter (zeroed before the launch)
    int* err;                     // raised when a wait gives up
};
// blocks of kWaveRows rows of an H-row image
int wave_blocks(int H);
// per frame of a batch, the caller provides the rings between its row blocks
// (wave_ring_cols columns each: kWaveRing when every block of the frame is
// resident at once, i.e. wave_blocks(H) <= cap, else a whole row, so that no
// block waits on the block below it) -- path costs first, the scalars at
// *scal_off -- and zeroed flag words (wave_flag_bytes)
int wave_ring_cols(int W, int H, int cap);
size_t wave_ring_bytes(int W, int H, int cap, size_t* scal_off);
size_t wave_flag_bytes(int H);
// CTAs of the two-pass kernels resident at once on the device (0: no
// cooperative launch)
int wave_capacity(int device);
// pass 0 or 1 with `ctas` persistent CTAs (at most wave_capacity), launched
// cooperatively; b.ticket[pass] must be zero
void launch_sgm_wave(const WaveBatch& b, int pass, int ctas, cudaStream_t st);

// Sbar may hold nparts partial sums, part_stride elements apart (summed here);
// pstride / bstride / bshift as in CostArgs (pstride 0: the [H][W][Ds] layout)
void launch_wta_refine(const uint16_t* Sbar, const int32_t* lo, int W, int H, int D, int Ds, int G,
                       const float* delta, Intr K, const float n[3], float* depth, int32_t* gwin,
                       cudaStream_t st, int nparts = 1, size_t part_stride = 0, size_t pstride = 0,
                       size_t bstride = 0, int bshift = 3);
// post-filters (Sec. 2.6): DoG mask (Alg. 3; 1 = enough texture, scratch:
// tmp W*H bytes, parent / size W*H ints, err one int set on a capped walk),
// estimates zeroed where the mask is 0, and the geometric consistency check
// (Alg. 4) zeroing pixels with fewer than eta_h hits
struct DogWeights { int32_t w[7]; };
void launch_dog_mask(const uint8_t* img, int W, int H, int pitch, const DogWeights& dw, uint8_t* mask, uint8_t* tmp,
                     int* parent, int* size, int* err, cudaStream_t st);
void launch_apply_mask(const uint8_t* mask, int W, int H, float* depth, float* normal, float* conf, cudaStream_t st);
struct GeoArgs {
    int W, H, n, eta_h;
    double fx, fy, cx, cy, eta_r;
    const float* dk[kMaxViews];
    double R[kMaxViews][9], t[kMaxViews][3];   // reference -> map k
};
void launch_geo_filter(const GeoArgs& g, float* depth, float* normal, float* conf, uint8_t* hits, cudaStream_t st);
void launch_delta_table(double rho0, double drho, int G, float* delta, cudaStream_t st);
// cost volume [Ds / 16][np][16] (as the batched cost kernel writes it) ->
// [np][Ds] (as the aggregation reads it); Ds a multiple of 16
void launch_relayout16(const uint16_t* src, uint16_t* dst, size_t np, int Ds, cudaStream_t st);
// out[i] = sum over p < parts of Sbar[p * stride + i] (the aggregate of a debug capture)
void launch_sum_parts(const uint16_t* Sbar, int parts, size_t stride, size_t n, uint16_t* out, cudaStream_t st);
void launch_median5(const float* in, int W, int H, float* out, cudaStream_t st);
void launch_normals(const float* depth, const uint8_t* img, int img_pitch, int W, int H, Intr K,
                    int radius, float beta, float* raw, float* normal, const float npl[3],
                    float rho_deg, float* conf, cudaStream_t st);
void launch_window(const float* dc, int Wc, int Hc, int W, int H, Intr K, const float n[3],
                   float rho0, float drho, int G, int D, int32_t* lo, cudaStream_t st);
void launch_dsn(const float* dc, const float* nc, int Wc, int Hc, int W, int H, Intr K, const float m[3],
                float drho, int dmax, int8_t* dI, cudaStream_t st);

// Records the thread-local error text returned by fassmvs_last_error(NULL).
void set_error(const char* msg);

// Counts kernel launches issued by this library (process-wide).
uint64_t launches();
void count_launch(int n = 1);

}  // namespace fm
