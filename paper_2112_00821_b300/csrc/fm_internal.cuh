// Internal declarations shared by the kernels and the C-ABI layer of the
// B300 FaSS-MVS library.  Nothing here is part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fm {

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
};
constexpr int kStageBX = 128, kStageBY = 80;
void launch_cost(const CostArgs& a, cudaStream_t st);
// multi-frame form: items[i] = (frame, tile x, tile y, chunk | chunks << 16);
// ctas > 0 persistent CTAs pulling items from *counter, else one CTA per item;
// ncc: every frame's args use the NCC cost (else the census)
void launch_cost_batch(const CostArgs* args, const int4* items, int n_items, int* counter, int ctas, bool ncc,
                       cudaStream_t st);
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
