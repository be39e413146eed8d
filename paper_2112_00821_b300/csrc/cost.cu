// Plane-sweep census cost volume (Alg. 1 of FaSS-MVS) for sm_103a.
//
// A CTA of 8 warps owns a 56 x 28 tile of reference pixels and walks every
// plane its windows need, one (plane, view) pair per iteration:
//   1. sampling: the 64 x 34 warped sample tile (tile + 9x7 census halo) is
//      produced cooperatively -- each warp owns 4 or 5 sample rows, each
//      lane two sample columns, the view image's taps read from a box staged
//      in shared memory by TMA; the homography's rows are stepped down the
//      column in double-float arithmetic, the position's nearest pixel comes
//      from an FP32 quotient q and its offset from the double-float residual
//      N - q D, so it is accurate to ~1e-7 px; the value is the bilinear
//      blend in lerp form about the nearest pixel in FP32, unrounded; a
//      lane's two columns go through packed FP32x2 operations, and the
//      stepping's set-up comes from the planning warp (warp 7), which has no
//      census and computes it for the pair two ahead while the others count;
//   2. one __syncthreads (the sample tile is double-buffered);
//   3. census: warp w < 7 takes columns 8w .. 8w + 7 of the tile, lane l
//      column 8w + l % 8 and rows 7 (l / 8) .. + 6 (every lane of the seven
//      warps busy; rows 72 words apart so the four row chunks fall in
//      different shared-memory banks); each comparison [V(q) < V(p)] is
//      decided on 2^15 (V(q) - V(p)) in FP32, whose sign and whether it
//      reaches 2 are funnel-shifted into four words per pixel; the XOR of the
//      sign bits with the reference census (pre-arranged in the same bit
//      order) and four popcounts give the Hamming distance, and the near ties
//      are decided exactly (see the exact census below); left / right sums
//      accumulate in registers over the views and the plane's costs are
//      stored after the last view.
// Seven-row chunks keep the census loop's unrolled code small enough for the
// instruction cache (13-row chunks on 56 x 52 tiles, with fewer halo samples,
// measured 8-14 % slower).
// Sampling reading (Alg. 1, shared with the oracle): the value of the
// neighbour image at the unrounded position H q, bilinear in lerp form,
// positions clamped to the image.
#include <type_traits>

#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int PW = 56, PH = 28;          // pixel tile
constexpr int SW = 72, SH = PH + 6;      // sample tile rows: 64 samples (PW + 8) in a 72-word stride
constexpr int NWARP = 8, THREADS = 256;
constexpr int CH = 7;                    // pixel rows per census chunk (PH / 4)
static_assert(PH == 4 * CH, "four census chunks per tile column");
constexpr int kCensusWarps = PW / 8;     // 7 warps x (8 columns x 4 chunks of 7 rows)
constexpr int kPlanWarp = NWARP - 1;     // plans and issues the staging copies
// first sample row of warp w's share (4 or 5 rows each)
__host__ __device__ constexpr int row_start(int w) { return (SH * w) / NWARP; }
constexpr int kMaxRows = 8;              // the largest share
static_assert(row_start(NWARP) - row_start(NWARP - 1) <= kMaxRows, "row shares");
constexpr float MAGIC = 12582912.0f;     // 1.5 * 2^23: adding it leaves an integer in the mantissa
constexpr int MAGIC_BITS = 0x4B400000;
constexpr int BYTE_BITS = 0x4B000000;    // 2^23 + b as a float, for a byte b
constexpr float TWO23 = 8388608.0f;

struct SmemCost {
    uint64_t mbar[2];                    // staging: completion of the tensor copy into slot 0 / 1
    int stg_x0[2], stg_y0[2], stg_ok[2]; // staging: box origin in the view image, and whether it was issued
    int stg_in[2];                       // staging: every sample of the pair maps 2 px or more inside the image
    int stg_dead;                        // a staged copy missed its bound: no further staging in this CTA
    float val[2][SH][SW];                // warped values minus 128 (FP32, unrounded)
    uint32_t okm[2][PH][2];              // centre-in-image bit per pixel column
    float hdf[2][18];                    // census: the pair's homography (high, low words), for near ties
    // the pair's set-up of the stepping, written by the planning warp two
    // pairs ahead: per lane the column terms h x of its two columns (U, V, D
    // as packed high / low words), per sampling warp the row term of its first
    // row, and the row steps
    float4 xt[2][3][32];
    float2 yt[2][NWARP][3];
    float2 st[2][3];
    uint32_t rkb[2][SH][2];              // census: risky samples, one bit per sample (columns 0-31, 32-63)
    uint8_t rkcol[2][NWARP][64];         // census: per sampling warp and pixel column, its rows whose
                                         // window columns hold a risky sample (one bit per row)
    union {
        uint4 refl[PH][PW];              // census: reference census in the comparison words' sign bits
        struct {
            float refv[SH][SW];          // NCC: reference grey levels on the sample grid
            int2 refs[PH][PW];           // NCC: (sum a, 25 sum a^2 - (sum a)^2) of each 5x5 window
        } ncc;
    };
    int32_t lo[PH][PW];
    int32_t rlo[PH], rhi[PH];            // per pixel row: planes its windows need, [rlo, rhi)
    int glo, ghi;
    int rskip;                           // tile rows the tile row above covers (computed, not stored)
};

struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a + b; the low word is not renormalised (it stays far below the high word
// over the few dozen steps of a column)
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}

// Values whose high word lies on the 2^-10 grid with magnitude below 2^12
// add exactly in FP32, so stepping down a column costs two additions
// (grid_add2: one packed addition per word for a lane's two columns): the
// homography is scaled (prep_level_kernel) so that |N|, |D| stay below 2^12
// over and well around the image, and the step's high words are on the grid.
constexpr float GRID_MAGIC = 12288.0f;   // 1.5 * 2^13: rounds |x| < 2^12 to the 2^-10 grid
__device__ __forceinline__ df to_grid(df a)
{
    float h = __fsub_rn(__fadd_rn(a.hi, GRID_MAGIC), GRID_MAGIC);
    return {h, __fadd_rn(a.lo, __fsub_rn(a.hi, h))};
}

// a * b for an integer-valued b (|b| < 2^24)
__device__ __forceinline__ df df_mul_int(df a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    float lo = __fmaf_rn(a.lo, b, e);
    float h = __fadd_rn(p, lo);
    return {h, __fsub_rn(lo, __fsub_rn(h, p))};
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ df load_df(const float* h, int i) { return {__ldg(h + i), __ldg(h + 9 + i)}; }

// The coordinates of a lane's two warped samples (columns lane and
// 32 + lane), each FP32 operation done once for both as a packed FP32x2
// operation (each half rounded as the scalar operation would round it).  For
// one coordinate, N / D is the position (D > 0); the arithmetic carries
// nr ~ -1 / D (one Newton step on the approximate reciprocal of -D, whose sign
// is that of its argument; nr = 0 for a point behind the camera, which then
// reads pixel 0 with weight 0, the clamped position of (-inf, -inf)), so that
// no packed operand is negated: nq = N.hi nr is minus the FP32 quotient
// q = N.hi / D, and the residual e = N - q D of the whole numerator (formed
// with fused multiply-adds, exact to far below an ulp of q) gives the
// position as q + e / D in double-float.  With c the integer nearest q, the
// offset f = (q - c) + e / D (the difference exact, one rounding in the fused
// multiply-add) is accurate to half an ulp of f: 1.5e-8 px, 3e-8 where the
// position lies within |N.lo / D| plus an ulp of q of a half integer and |f|
// passes 1/2.  Every value is the exact negation of the one the positive form
// would round (round-to-nearest is symmetric).  The bilinear blend weighs
// pixel c and its neighbour c + s (s = the sign of f) with |f| < 1, so it
// interpolates between them and never extrapolates (a floor-based cell
// would, by up to that error times the change of slope across the cell
// edge); a position outside the image reads the nearest image pixel with
// weight 0, its clamp.
//
// The nearest pixel, neighbour steps and weights of one warped sample.
struct SPos { int iu, iv, su, sv; float a, b; };

struct df2 { float2 hi, lo; };
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ df2 grid_add2(df2 a, df2 b) { return {__fadd2_rn(a.hi, b.hi), __fadd2_rn(a.lo, b.lo)}; }

// The per-warp set-up of the stepping for the lane's two columns, packed as
// above: df_mul_int, df_add with a term shared by both columns, and to_grid,
// each half equal to the scalar function's result bit for bit (y - x is
// formed as fma(x, -1, y), one rounding of the exact difference; -a.hi is
// passed in so that no packed operand is negated).
__device__ __forceinline__ df2 df_mul_int2(df a, float na_hi, float2 b)
{
    const float2 np = __fmul2_rn(f2(na_hi), b);                    // -p
    const float2 e = __ffma2_rn(f2(a.hi), b, np);
    const float2 lo = __ffma2_rn(f2(a.lo), b, e);
    const float2 h = __ffma2_rn(np, f2(-1.0f), lo);                // p + lo
    const float2 t = __fadd2_rn(h, np);                            // h - p
    return {h, __ffma2_rn(t, f2(-1.0f), lo)};
}
__device__ __forceinline__ df2 df_add2(df2 a, df b)
{
    const float2 bh = f2(b.hi);
    const float2 s = __fadd2_rn(a.hi, bh);
    const float2 bb = __ffma2_rn(a.hi, f2(-1.0f), s);              // s - a
    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, f2(-1.0f), s), f2(-1.0f), a.hi),
                                __ffma2_rn(bb, f2(-1.0f), bh));    // (a - (s - bb)) + (b - bb)
    return {s, __fadd2_rn(e, __fadd2_rn(a.lo, f2(b.lo)))};
}
__device__ __forceinline__ df2 to_grid2(df2 a)
{
    const float2 h = __fadd2_rn(__fadd2_rn(a.hi, f2(GRID_MAGIC)), f2(-GRID_MAGIC));
    return {h, __fadd2_rn(a.lo, __ffma2_rn(h, f2(-1.0f), a.hi))};
}

// a pair whose whole tile maps 2 px or more inside the image: no clamping
struct Coord2 { int i0, i1, s0, s1; float2 w; };
__device__ __forceinline__ Coord2 coord2_in(df2 N, df2 D, float2 nr)
{
    const float2 nq = __fmul2_rn(N.hi, nr);
    const float2 e = __ffma2_rn(nq, D.lo, __fadd2_rn(__ffma2_rn(nq, D.hi, N.hi), N.lo));
    // -c = rint(-q); -f = e nr + (-q - (-c))
    const float2 nc = make_float2(rintf(nq.x), rintf(nq.y));
    const float2 nf = __ffma2_rn(e, nr, __ffma2_rn(nc, f2(-1.0f), nq));
    const float2 cm = __fadd2_rn(nc, f2(MAGIC));
    return {MAGIC_BITS - __float_as_int(cm.x), MAGIC_BITS - __float_as_int(cm.y), nf.x > 0.0f ? -1 : 1,
            nf.y > 0.0f ? -1 : 1, make_float2(fabsf(nf.x), fabsf(nf.y))};
}

struct SPos2 { int iu0, iv0, su0, sv0, iu1, iv1, su1, sv1; float2 a, b; };
__device__ __forceinline__ SPos2 sample_pos2_in(df2 Nu, df2 Nv, df2 Dn)
{
    const float2 dsum = __fadd2_rn(Dn.hi, Dn.lo);
    const float2 nr0 = make_float2(rcp_approx(-dsum.x), rcp_approx(-dsum.y));
    const float2 nr = __ffma2_rn(nr0, __ffma2_rn(dsum, nr0, f2(1.0f)), nr0);
    const Coord2 cu = coord2_in(Nu, Dn, nr);
    const Coord2 cv = coord2_in(Nv, Dn, nr);
    return {cu.i0, cv.i0, cu.s0, cv.s0, cu.i1, cv.i1, cu.s1, cv.s1, cu.w, cv.w};
}

// Any pair (the clamped reading): -q is clamped to [-size, 1] before the
// rounding (so q to [-1, size], a NaN to -1), and per half: the nearest pixel
// clamped to the image, no neighbour step (weight 0) where the pixel or its
// neighbour leaves the image, and in = the position lies on [0, size - 1].
// For a position 2 px or more inside the image it gives what coord2_in
// gives.
__device__ __forceinline__ void coord_fix(int ci, float nf, int maxi, int& i, int& s, float& w, bool& in)
{
    const bool neg = nf > 0.0f;                           // f < 0
    const int nb = neg ? ci - 1 : ci + 1;
    const int cc = min(max(ci, 0), maxi);
    const bool edge = cc != ci || (unsigned)nb > (unsigned)maxi;
    in = (unsigned)ci <= (unsigned)maxi && !(ci == 0 && neg) && !(ci == maxi && nf < 0.0f);
    i = cc;
    s = edge ? 0 : (neg ? -1 : 1);
    w = edge ? 0.0f : fabsf(nf);
}
__device__ __forceinline__ Coord2 coord2_clamped(df2 N, df2 D, float2 nr, float maxf, int maxi, bool& in0, bool& in1)
{
    const float2 nq = __fmul2_rn(N.hi, nr);
    const float2 e = __ffma2_rn(nq, D.lo, __fadd2_rn(__ffma2_rn(nq, D.hi, N.hi), N.lo));
    const float lo = -(maxf + 1.0f);
    const float2 nc = make_float2(rintf(fmaxf(fminf(nq.x, 1.0f), lo)), rintf(fmaxf(fminf(nq.y, 1.0f), lo)));
    const float2 nf = __ffma2_rn(e, nr, __ffma2_rn(nc, f2(-1.0f), nq));
    const float2 cm = __fadd2_rn(nc, f2(MAGIC));
    Coord2 o;
    coord_fix(MAGIC_BITS - __float_as_int(cm.x), nf.x, maxi, o.i0, o.s0, o.w.x, in0);
    coord_fix(MAGIC_BITS - __float_as_int(cm.y), nf.y, maxi, o.i1, o.s1, o.w.y, in1);
    return o;
}
// ok0 / ok1: the sample's position lies on the image grid (and in front)
__device__ __forceinline__ SPos2 sample_pos2(float wm1, float hm1, df2 Nu, df2 Nv, df2 Dn, bool& ok0, bool& ok1)
{
    const float2 dsum = __fadd2_rn(Dn.hi, Dn.lo);
    const float2 nr0 = make_float2(rcp_approx(-dsum.x), rcp_approx(-dsum.y));
    float2 nr = __ffma2_rn(nr0, __ffma2_rn(dsum, nr0, f2(1.0f)), nr0);
    const bool f0 = dsum.x > 0.0f, f1 = dsum.y > 0.0f;
    nr = make_float2(f0 ? nr.x : 0.0f, f1 ? nr.y : 0.0f);
    bool iu0, iu1, iv0, iv1;
    const Coord2 cu = coord2_clamped(Nu, Dn, nr, wm1, (int)wm1, iu0, iu1);
    const Coord2 cv = coord2_clamped(Nv, Dn, nr, hm1, (int)hm1, iv0, iv1);
    ok0 = f0 && iu0 && iv0;
    ok1 = f1 && iu1 && iv1;
    return {cu.i0, cv.i0, cu.s0, cv.s0, cu.i1, cv.i1, cu.s1, cv.s1, cu.w, cv.w};
}

// 2^23 + b as a float for a byte b (exact)
__device__ __forceinline__ float bf(int b) { return __int_as_float(BYTE_BITS + b); }

// bilinear blend in lerp form about the nearest pixel: top = I0 + a (Iu - I0)
// along u, bottom likewise one row towards the position, value = top + b
// (bottom - top) -- the usual bilinear value.  The values are carried minus
// 128 (the byte differences and the shifted taps are exact), which halves
// their magnitude and so their rounding error; the census compares
// differences and the NCC deviations from the window mean, so the shift
// changes no result.
constexpr float VBIAS = TWO23 + 128.0f;
// pl: the four taps are equal (a plateau sample: its value is that integer, exactly)
__device__ __forceinline__ float blend(int i0, int iu, int iv, int iuv, float a, float b, bool& pl)
{
    const float t0 = bf(i0), tv = bf(iv);
    const float d0 = __fsub_rn(bf(iu), t0), d1 = __fsub_rn(bf(iuv), tv);
    pl = d0 == 0.0f && d1 == 0.0f && t0 == tv;
    const float top = __fmaf_rn(a, d0, __fsub_rn(t0, VBIAS));
    const float bot = __fmaf_rn(a, d1, __fsub_rn(tv, VBIAS));
    return __fmaf_rn(b, __fsub_rn(bot, top), top);
}

// the taps from global memory
__device__ __forceinline__ float taps_global(const uint8_t* __restrict__ img, int pitch, int W, int H, SPos p,
                                             bool& pl)
{
    if (!FM_IN(p.iu, W, 0x102) || !FM_IN(p.iu + p.su, W, 0x102) || !FM_IN(p.iv, H, 0x102) ||
        !FM_IN(p.iv + p.sv, H, 0x102)) {
        pl = false;
        return 0.0f;
    }
    const uint8_t* r0 = img + (size_t)p.iv * pitch + p.iu;
    const int dv = p.sv * pitch;
    return blend(__ldg(r0), __ldg(r0 + p.su), __ldg(r0 + dv), __ldg(r0 + dv + p.su), p.a, p.b, pl);
}

// the taps from the staged box whose origin is (sx0, sy0) (in_box true)
__device__ __forceinline__ float taps_staged(const uint8_t* stg, int sx0, int sy0, SPos p, bool& pl)
{
    const int o = (p.iv - sy0) * kStageBX + (p.iu - sx0);
    const int dv = p.sv * kStageBX;
    if (!FM_IN(o + min(p.su, 0) + min(dv, 0), kStageBX * kStageBY, 0x101) ||
        !FM_IN(o + max(p.su, 0) + max(dv, 0), kStageBX * kStageBY, 0x101)) {
        pl = false;
        return 0.0f;
    }
    const uint8_t* r0 = stg + o;
    return blend(r0[0], r0[p.su], r0[dv], r0[dv + p.su], p.a, p.b, pl);
}

// the two samples of a lane from the staged box (interior pairs: the
// footprints lie in it), blended as blend() does, as FP32x2 pairs: the tap
// differences and the lerps are single roundings of the same operands
__device__ __forceinline__ float2 taps2_staged(const uint8_t* stg, int sx0, int sy0, const SPos2& p, bool& pl0,
                                               bool& pl1)
{
    const int o0 = (p.iv0 - sy0) * kStageBX + (p.iu0 - sx0), dv0 = p.sv0 * kStageBX;
    const int o1 = (p.iv1 - sy0) * kStageBX + (p.iu1 - sx0), dv1 = p.sv1 * kStageBX;
    if (!FM_IN(o0 + min(p.su0, 0) + min(dv0, 0), kStageBX * kStageBY, 0x101) ||
        !FM_IN(o0 + max(p.su0, 0) + max(dv0, 0), kStageBX * kStageBY, 0x101) ||
        !FM_IN(o1 + min(p.su1, 0) + min(dv1, 0), kStageBX * kStageBY, 0x101) ||
        !FM_IN(o1 + max(p.su1, 0) + max(dv1, 0), kStageBX * kStageBY, 0x101)) {
        pl0 = pl1 = false;
        return make_float2(0.0f, 0.0f);
    }
    const uint8_t* r0 = stg + o0;
    const uint8_t* r1 = stg + o1;
    const int a0 = r0[0], au = r0[p.su0], av = r0[dv0], auv = r0[dv0 + p.su0];
    const int b0 = r1[0], bu = r1[p.su1], bv = r1[dv1], buv = r1[dv1 + p.su1];
    pl0 = ((a0 ^ au) | (av ^ auv) | (a0 ^ av)) == 0;
    pl1 = ((b0 ^ bu) | (bv ^ buv) | (b0 ^ bv)) == 0;
    const float2 t0 = make_float2(bf(a0), bf(b0)), tv = make_float2(bf(av), bf(bv));
    const float2 d0 = __ffma2_rn(t0, f2(-1.0f), make_float2(bf(au), bf(bu)));
    const float2 d1 = __ffma2_rn(tv, f2(-1.0f), make_float2(bf(auv), bf(buv)));
    const float2 top = __ffma2_rn(p.a, d0, __fadd2_rn(t0, f2(-VBIAS)));
    const float2 bot = __ffma2_rn(p.a, d1, __fadd2_rn(tv, f2(-VBIAS)));
    return __ffma2_rn(p.b, __ffma2_rn(top, f2(-1.0f), bot), top);
}

// the 2x2 footprint lies in the staged box
__device__ __forceinline__ bool in_box(int sx0, int sy0, SPos p)
{
    return (unsigned)(p.iu + min(p.su, 0) - sx0) <= (unsigned)(kStageBX - 2) &&
           (unsigned)(p.iv + min(p.sv, 0) - sy0) <= (unsigned)(kStageBY - 2);
}

// ---------------------------------------------------------------- exact census
// A census comparison [V(q) < V(p)] is decided on the FP32 values (V = warped
// value - 128) by the sign of x = 2^15 (V(q) - V(p)), one rounding of an
// exact difference; bit 30 of x records |x| >= 2, i.e. |V(q) - V(p)| >= 2^-14,
// and a funnel shift by two keeps both bits.  An FP32 value lies within
// 2.7e-5 of the FP64 value of the sampling reading: each lerp's weight error
// (at most 3e-8 px) times a tap difference of at most 255, plus half an ulp of
// the top and bottom lerps (|value| < 128: 3.8e-6), of their difference
// (< 256: 7.6e-6, times the weight <= 1/2) and of the value, 1.14e-5 +
// 3.8e-6 + 7.6e-6 + 3.8e-6 (measured on whole 1080p pairs: at most 2.2e-5).
// Below 2^-15 = 3.05e-5, so a comparison whose FP32 difference reaches
// 2^-14 = 6.1e-5 has the FP64 comparison's sign.  The
// others -- near ties -- are decided again: equal values of one reference
// position are ties in FP64 as well; a pixel whose centre is an integer and
// whose window holds no risky sample (a non-plateau value within 2^-13 of an
// integer) has only ties between plateaus of equal pixels, which are exact
// integers in FP64 too, and skips the step; the rest are recomputed in
// double-float from the homography and the image (cen_fix).
constexpr float kCensusScale = 32768.0f;
constexpr float kRiskyBound = 0x1p-13f;
//
// The 62 comparisons of a pixel, in window order k = 9 dy + dx (k = 31, the
// centre, skipped), go to four words: k 0-15, 16-30, 32-47, 48-62.
__host__ __device__ constexpr int cword(int k) { return k < 16 ? 0 : (k < 31 ? 1 : (k < 48 ? 2 : 3)); }
__host__ __device__ constexpr int cbase(int w) { return w == 0 ? 0 : (w == 1 ? 16 : (w == 2 ? 32 : 48)); }
__host__ __device__ constexpr int ccount(int w) { return (w & 1) ? 15 : 16; }
// bit of the sign of comparison k in its word (the big-difference bit is one below)
__host__ __device__ constexpr int cbit(int k) { return 2 * (ccount(cword(k)) - 1 - (k - cbase(cword(k)))) + 1; }
constexpr uint32_t SIGN_BITS = 0xAAAAAAAAu;
__host__ __device__ constexpr uint32_t big_bits(int w) { return (w & 1) ? 0x15555555u : 0x55555555u; }

// The big-difference bits (in word w) of the comparisons that a pixel on
// image edges makes with itself: window position k = 9 (dy + 3) + dx + 4
// clamps back onto the pixel when each offset is zero or points out of the
// image across an edge the pixel lies on (L, R: left, right column; T, B: top,
// bottom row).  Those comparisons are ties in FP64 as in FP32, so they are
// left out of the near ties.
__host__ __device__ constexpr uint32_t self_mask(int w, bool L, bool R, bool T, bool B)
{
    uint32_t m = 0;
    for (int k = 0; k < 63; ++k) {
        if (k == 31 || cword(k) != w) continue;
        const int dy = k / 9 - 3, dx = k % 9 - 4;
        const bool xs = dx == 0 || (L && dx < 0) || (R && dx > 0);
        const bool ys = dy == 0 || (T && dy < 0) || (B && dy > 0);
        if (xs && ys) m |= 1u << (cbit(k) - 1);
    }
    return m;
}
constexpr uint32_t kSelfLeft = self_mask(1, true, false, false, false);    // dy = 0, dx = -4 .. -1
constexpr uint32_t kSelfRight = self_mask(2, false, true, false, false);   // dy = 0, dx = 1 .. 4
static_assert(self_mask(0, false, false, false, false) == 0u && self_mask(3, true, true, false, false) == 0u,
              "a pixel inside the image has no self comparisons");

// canonical 9x7 census word -> the sign bits of the four comparison words
__device__ __forceinline__ uint4 to_layout(uint64_t c)
{
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 63; ++k) {
        if (k == 31) continue;
        w[cword(k)] |= (uint32_t)((c >> k) & 1u) << cbit(k);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---- double-float evaluation of one warped sample, for the near ties
__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// N / D for D > 0 (a few ulps of double-float)
__device__ __forceinline__ df df_div(df N, df D)
{
    const float r0 = rcp_approx(D.hi);
    const float r = __fmaf_rn(r0, __fmaf_rn(-D.hi, r0, 1.0f), r0);
    const float qh = __fmul_rn(N.hi, r);
    const df p = two_prod(qh, D.hi);
    const float rem = __fadd_rn(__fsub_rn(__fsub_rn(N.hi, p.hi), p.lo), __fsub_rn(N.lo, __fmul_rn(qh, D.lo)));
    return two_sum(qh, __fmul_rn(rem, r));
}

// (hi, lo) with |lo| <= half an ulp of hi.  The products below drop the
// low-times-low term, which is negligible only for normalised operands: the
// offset left by subtracting the floor keeps few significant bits in its high
// word, and its unnormalised low word times that of a tap difference reached
// 2e-8 grey levels, enough to misorder a near tie.
__device__ __forceinline__ df df_norm(df a) { return two_sum(a.hi, a.lo); }

// the cell (clamped to [0, cmax]) and offset (clamped to [0, 1], normalised)
// of a position u in double-float
__device__ __forceinline__ int df_cell(df u, int cmax, df& a)
{
    float fl = floorf(u.hi);
    df f = {__fsub_rn(u.hi, fl), u.lo};                     // the first word exact
    if (__fadd_rn(f.hi, f.lo) < 0.0f) { fl = __fsub_rn(fl, 1.0f); f.hi = __fadd_rn(f.hi, 1.0f); }
    else if (__fadd_rn(f.hi, f.lo) >= 1.0f) { fl = __fadd_rn(fl, 1.0f); f.hi = __fsub_rn(f.hi, 1.0f); }
    if (fl < 0.0f) { a = {0.0f, 0.0f}; return 0; }
    if (fl > (float)cmax) { a = {1.0f, 0.0f}; return cmax; }
    a = df_norm(f);
    return (int)fl;
}

// t0 + a (t1 - t0) for taps t0, t1 and a normalised double-float offset a
// (normalised result)
__device__ __forceinline__ df df_lerp_taps(float t0, float t1, df a)
{
    const float d = __fsub_rn(t1, t0);
    const df p = two_prod(a.hi, d);
    const df s = two_sum(t0, p.hi);
    return df_norm({s.hi, __fadd_rn(s.lo, __fadd_rn(p.lo, __fmul_rn(a.lo, d)))});
}

// value - 128 of the warped neighbour k at reference pixel (X, Y) under the
// homography h (18 floats: the high then the low words of the nine entries),
// in double-float arithmetic: the position to ~1e-11 px, every product taken
// on normalised operands, so the value of the sampling reading to ~1e-11 grey
// levels
__device__ __forceinline__ df sample_exact(const CostArgs& a, const float* h, int k, int X, int Y)
{
    const float fx = (float)X, fy = (float)Y;
    auto e = [&](int i) { return df{h[i], h[9 + i]}; };
    const df N = df_add(df_add(df_mul_int(e(0), fx), df_mul_int(e(1), fy)), e(2));
    const df M = df_add(df_add(df_mul_int(e(3), fx), df_mul_int(e(4), fy)), e(5));
    const df D = df_add(df_add(df_mul_int(e(6), fx), df_mul_int(e(7), fy)), e(8));
    df au = {0.0f, 0.0f}, av = {0.0f, 0.0f};
    int iu = 0, iv = 0;
    if (__fadd_rn(D.hi, D.lo) > 0.0f) {
        iu = df_cell(df_div(N, D), a.W - 2, au);
        iv = df_cell(df_div(M, D), a.H - 2, av);
    }
    if (!FM_IN(iu, a.W - 1, 0x107) || !FM_IN(iv, a.H - 1, 0x107)) return {0.0f, 0.0f};
    const uint8_t* r0 = a.views.img[k] + (size_t)iv * a.pitch + iu;
    const float i00 = (float)__ldg(r0) - 128.0f, i01 = (float)__ldg(r0 + 1) - 128.0f;
    const float i10 = (float)__ldg(r0 + a.pitch) - 128.0f, i11 = (float)__ldg(r0 + a.pitch + 1) - 128.0f;
    const df top = df_lerp_taps(i00, i01, au), bot = df_lerp_taps(i10, i11, au);
    // top + b (bot - top)
    const df dd = df_norm(df_add(bot, {-top.hi, -top.lo}));
    const df p = two_prod(av.hi, dd.hi);
    const float pl = __fadd_rn(p.lo, __fadd_rn(__fmul_rn(av.hi, dd.lo), __fmul_rn(av.lo, dd.hi)));
    return df_add(top, {p.hi, pl});
}

// The correction to the FP32 Hamming distance of pixel (sample row j0 + 3,
// column c0 + 4) once its near ties -- the comparisons whose FP32 difference
// stays below 2^-14 -- are decided exactly, computed by the whole warp (lane l
// takes window positions l and l + 32; the same value returned in every
// lane).  Equal values of one reference position (a window clamped at the
// image border) are ties in FP64 as well, and so are equal integers of two
// samples that are not risky (rkb: an integer-valued sample that is not
// risky is a plateau); the rest are recomputed in double-float (a non-plateau
// value close to an integer can come out as that integer in FP32).  Sample
// rows past jlast (below the image) read row jlast, as the census does.
__device__ __forceinline__ int cen_fix(const CostArgs& a, const float (*vt)[SW], const uint32_t (*rkb)[2],
                                       const float* h, int k, int tx0, int ty0, int j0, int c0, int jlast, uint4 rf,
                                       int lane)
{
    const float vp = vt[min(j0 + 3, jlast)][c0 + 4];
    const bool rp = (rkb[min(j0 + 3, jlast)][(c0 + 4) >> 5] >> ((c0 + 4) & 31)) & 1u;
    const float cs = __fmul_rn(kCensusScale, vp);
    const int xp = min(max(tx0 + c0, 0), a.W - 1), yp = min(max(ty0 + j0, 0), a.H - 1);
    int delta = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int kk = lane + 32 * t;
        if (kk == 31 || kk >= 63) continue;
        const int dy = kk / 9, dx = kk - 9 * (kk / 9);
        if (!FM_IN(min(j0 + dy, jlast) * SW + c0 + dx, SH * SW, 0x10a)) continue;
        const float vq = vt[min(j0 + dy, jlast)][c0 + dx];
        const float x = __fmaf_rn(vq, kCensusScale, -cs);
        if (fabsf(x) >= 2.0f) continue;
        const int xq = min(max(tx0 - 4 + c0 + dx, 0), a.W - 1), yq = min(max(ty0 - 3 + j0 + dy, 0), a.H - 1);
        const bool rq = (rkb[min(j0 + dy, jlast)][(c0 + dx) >> 5] >> ((c0 + dx) & 31)) & 1u;
        if (vq == vp && ((xq == xp && yq == yp) || (vq == rintf(vq) && !rq && !rp))) continue;
        const df ep = sample_exact(a, h, k, xp, yp);
        const df eq = sample_exact(a, h, k, xq, yq);
        const df d = two_sum(eq.hi, -ep.hi);
        const float diff = __fadd_rn(d.hi, __fadd_rn(d.lo, __fsub_rn(eq.lo, ep.lo)));
        const uint32_t exact = diff < 0.0f ? 1u : 0u;
        const uint32_t fp = __float_as_uint(x) >> 31;
        if (exact != fp) {
            const int w = cword(kk);
            const uint32_t rw = w == 0 ? rf.x : (w == 1 ? rf.y : (w == 2 ? rf.z : rf.w));
            const uint32_t rb = (rw >> (2 * (ccount(w) - 1 - (kk - cbase(w))) + 1)) & 1u;
            delta += fp == rb ? 1 : -1;
        }
    }
    return __reduce_add_sync(0xFFFFFFFFu, delta);
}

// The near ties that the census's filter leaves (fmask: this lane's chunk
// rows, pixel rows pr0 + r at column pc), decided exactly by cen_fix, one
// pixel at a time for the whole warp; corr[r] gets the change of chunk row r's
// Hamming distance (zero for the others).  Called by the whole warp, and out
// of line: about one warp-pair in eighty has a pixel left here.
__device__ __noinline__ void fix_ties(const CostArgs& a, const SmemCost& sm, int buf, int k, int tx0, int ty0,
                                      int pr0, int pc, int jlast, uint32_t fmask, int lane, int* corr)
{
    const float(*vt)[SW] = sm.val[buf];
#pragma unroll
    for (int r = 0; r < CH; ++r) corr[r] = 0;
    uint32_t pend = __ballot_sync(0xFFFFFFFFu, fmask != 0u);
    while (pend) {
        const int src = __ffs(pend) - 1;
        const uint32_t fm = __shfl_sync(0xFFFFFFFFu, fmask, src);
        const int r = __ffs(fm) - 1;
        const int c0 = __shfl_sync(0xFFFFFFFFu, pc, src);
        const int j0 = __shfl_sync(0xFFFFFFFFu, pr0, src) + r;
        const int d = cen_fix(a, vt, sm.rkb[buf], sm.hdf[buf], k, tx0, ty0, j0, c0, jlast, sm.refl[j0][c0], lane);
        if (lane == src) {
            fmask &= fmask - 1u;
            corr[r] += d;
        }
        pend = __ballot_sync(0xFFFFFFFFu, fmask != 0u);
    }
}

// ---------------------------------------------------------------- staging
// For each (plane, view) pair one elected thread copies a kStageBX x kStageBY
// box of the view image that holds the warped sample tile into shared memory
// with a TMA tensor copy, one pair ahead of the sampling (two slots, the same
// parity as the sample-tile double buffer, so the loop's one barrier orders
// every reuse).  Samples whose 2x2 taps lie outside the box read global memory
// as before, so results never depend on the box.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_init(SmemCost& sm)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sm.mbar[i])), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.stg_dead = 0;
        sm.stg_ok[0] = sm.stg_ok[1] = 0;
        sm.stg_in[0] = sm.stg_in[1] = 0;
    }
    __syncthreads();
}

__device__ __forceinline__ void stage_issue(uint64_t* mbar, uint8_t* dst, const void* tmap, int x0, int y0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(mbar)), "r"(kStageBX * kStageBY)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)tmap), "r"(x0), "r"(y0), "r"(smem_u32(mbar))
        : "memory");
}

// waits for the phase of the given parity, at most `bound` clocks (2^31,
// about a second; 2^21 under the test hook); false when the bound is reached
__device__ __forceinline__ bool stage_wait(uint64_t* mbar, uint32_t parity, long long bound)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > bound) return false;
    }
}

// the planning warp: the box for pair (g, k) into `slot`.  Lanes 0-3 warp the four
// corners of the (clamped) sample tile in FP32 (the box gets two pixels of
// margin, more than the FP32 error of a corner); all four must lie in front of
// the view.  The box origin's x is a multiple of 16 (TMA alignment).
__device__ __forceinline__ void stage_plan(const CostArgs& a, SmemCost& sm, uint8_t* stg, int tx0, int ty0, int g,
                                           int k, int slot, int lane)
{
    float u = 0.0f, v = 0.0f;
    bool front = true;
    if (lane < 4) {
        const float* h = a.htab + ((size_t)g * a.V + k) * 18;
        float hh[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) hh[i] = __ldg(h + i) + __ldg(h + 9 + i);
        const float x = (float)((lane & 1) ? min(max(tx0 + 59, 0), a.W - 1) : min(max(tx0 - 4, 0), a.W - 1));
        const float y = (float)((lane & 2) ? min(max(ty0 + PH + 2, 0), a.H - 1) : min(max(ty0 - 3, 0), a.H - 1));
        const float nu = hh[0] * x + hh[1] * y + hh[2];
        const float nv = hh[3] * x + hh[4] * y + hh[5];
        const float dn = hh[6] * x + hh[7] * y + hh[8];
        front = dn > 0.0f;
        if (front) {
            u = nu / dn;
            v = nv / dn;
        }
    }
    const bool all_front = __all_sync(0xFFFFFFFFu, front);
    float umin = lane < 4 ? u : 3.0e38f, umax = lane < 4 ? u : -3.0e38f;
    float vmin = lane < 4 ? v : 3.0e38f, vmax = lane < 4 ? v : -3.0e38f;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        umin = fminf(umin, __shfl_xor_sync(0xFFFFFFFFu, umin, o));
        umax = fmaxf(umax, __shfl_xor_sync(0xFFFFFFFFu, umax, o));
        vmin = fminf(vmin, __shfl_xor_sync(0xFFFFFFFFu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, o));
    }
    if (lane == 0) {
        int ok = 0, x0 = 0, y0 = 0, in = 0;
        if (all_front && !sm.stg_dead) {
            const float wm = (float)(a.W - 1), hm = (float)(a.H - 1);
            const float ulo = fminf(fmaxf(umin, 0.0f), wm), uhi = fminf(fmaxf(umax, 0.0f), wm);
            const float vlo = fminf(fmaxf(vmin, 0.0f), hm), vhi = fminf(fmaxf(vmax, 0.0f), hm);
            x0 = max((int)floorf(ulo) - 2, 0) & ~15;
            y0 = max((int)floorf(vlo) - 2, 0);
            ok = (int)floorf(uhi) + 3 <= x0 + kStageBX - 1 && (int)floorf(vhi) + 3 <= y0 + kStageBY - 1;
            // a rectangle in front of the camera maps onto the convex hull of
            // its corners' images, so with a corner error far below a pixel
            // every sample of the pair then lies in [1, size - 2] with its
            // neighbour taps, all inside the box
            in = ok && umin >= 2.0f && vmin >= 2.0f && umax <= (float)(a.W - 3) && vmax <= (float)(a.H - 3);
        }
        sm.stg_x0[slot] = x0;
        sm.stg_y0[slot] = y0;
        sm.stg_ok[slot] = ok;
        sm.stg_in[slot] = in;
        if (ok && !a.stage_test)
            stage_issue(&sm.mbar[slot], stg + slot * kStageBX * kStageBY,
                        static_cast<const char*>(a.tmaps) + (size_t)k * 128, x0, y0);
    }
}

// The planning warp: the set-up of pair (g, k)'s stepping into `slot` (see
// SmemCost::xt), which the sampling warps combine exactly as they would
// compute it themselves.  (The pair's homography for the near-tie recompute,
// hdf, is read during the census while this runs for the pair two ahead: the
// sampling warps keep storing it.)
__device__ __forceinline__ void stage_setup(const CostArgs& a, SmemCost& sm, int tx0, int ty0, int g, int k,
                                            int slot, int lane)
{
    const float* h = a.htab + ((size_t)(FM_IN(g, a.G, 0x108) ? g : 0) * a.V + k) * 18;
    // column terms of columns lane and 32 + lane
    const int W = a.W, H = a.H;
    const float2 fx = make_float2((float)min(max(tx0 - 4 + lane, 0), W - 1), (float)min(max(tx0 + 28 + lane, 0), W - 1));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const df hc = load_df(h, 3 * c);
        const df2 x = df_mul_int2(hc, -hc.hi, fx);
        sm.xt[slot][c][lane] = make_float4(x.hi.x, x.hi.y, x.lo.x, x.lo.y);
    }
    // row term of warp w's first row (lane 3 w + c), and the row steps
    if (lane < 3 * NWARP) {
        const int w = lane / 3, c = lane - 3 * w;
        const float fy = (float)min(max(ty0 - 3 + row_start(w), 0), H - 1);
        const df y = df_add(df_mul_int(load_df(h, 3 * c + 1), fy), load_df(h, 3 * c + 2));
        sm.yt[slot][w][c] = make_float2(y.hi, y.lo);
    }
    if (lane < 3) {
        const df s = to_grid(load_df(h, 3 * lane + 1));
        sm.st[slot][lane] = make_float2(s.hi, s.lo);
    }
}

// One tile (bx, by) of one frame, plane chunk bz of nz, with the census (NCC
// false) or NCC 5x5 cost.  Called by the single-frame grid kernel and by the
// multi-frame kernel, both with their arguments in shared memory.
template <bool NCC, bool DBG>
__device__ __forceinline__ void cost_tile(const CostArgs& a, int bx, int by, int bz, int nz, SmemCost& sm,
                                          uint8_t* stg, uint32_t& phase)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the last tile row ends on the image's last row (for an image at least a
    // tile high), so that row is chunk row CH - 1 of the last chunk; its rows
    // above by * PH, which the tile row above covers, are computed but not
    // stored
    const int tx0 = bx * PW, ty0 = a.H >= PH ? min(by * PH, a.H - PH) : 0;
    const int W = a.W, H = a.H;

    if (tid == 0) { sm.glo = a.G; sm.ghi = 0; sm.rskip = by * PH - ty0; }
    __syncthreads();
    for (int i = tid; i < PH * PW; i += THREADS) {
        const int r = i / PW, c = i % PW;
        const int px = tx0 + c, py = ty0 + r;
        const bool in = px < W && py < H;
        const int l = in ? (a.lo ? a.lo[(size_t)py * W + px] : 0) : (1 << 30);
        sm.lo[r][c] = l;
        if (in) {
            atomicMin(&sm.glo, l);
            atomicMax(&sm.ghi, l + a.D);
        }
        if constexpr (!NCC) sm.refl[r][c] = to_layout(in ? a.cref[(size_t)py * W + px] : 0ull);
    }
    // the window map and the tile's plane range are read below by every thread
    __syncthreads();
    if constexpr (NCC) {
        // reference values on the sample grid (clamp-to-edge), then each pixel's
        // 5x5 window sums (exact integers)
        for (int i = tid; i < SH * SW; i += THREADS) {
            const int j = i / SW, c = i % SW;
            const uint8_t* row = a.ref + (size_t)min(max(ty0 - 3 + j, 0), H - 1) * a.ref_pitch;
            sm.ncc.refv[j][c] = (float)__ldg(row + min(max(tx0 - 4 + c, 0), W - 1));
        }
        __syncthreads();
        for (int i = tid; i < PH * PW; i += THREADS) {
            const int r = i / PW, c = i % PW;
            int sa = 0, saa = 0;
#pragma unroll
            for (int dy = 0; dy < 5; ++dy)
#pragma unroll
                for (int dx = 0; dx < 5; ++dx) {
                    const int v = (int)sm.ncc.refv[r + 1 + dy][c + 2 + dx];
                    sa += v;
                    saa += v * v;
                }
            sm.ncc.refs[r][c] = make_int2(sa, 25 * saa - sa * sa);
        }
    }
    // per pixel row, the planes its windows need; empty sample buffers, so
    // that a row no warp sampled yet holds finite values
    for (int r = tid; r < PH; r += THREADS) {
        int l = a.G, h = 0;
        for (int c = 0; c < PW; ++c) {
            const int v = sm.lo[r][c];
            if (v != (1 << 30)) {
                l = min(l, v);
                h = max(h, v + a.D);
            }
        }
        sm.rlo[r] = l;
        sm.rhi[r] = h;
    }
    for (int i = tid; i < 2 * SH * SW; i += THREADS) (&sm.val[0][0][0])[i] = 0.0f;
    for (int i = tid; i < 2 * PH * 2; i += THREADS) (&sm.okm[0][0][0])[i] = 0u;
    for (int i = tid; i < 2 * SH * 2; i += THREADS) (&sm.rkb[0][0][0])[i] = 0u;
    // planes of this tile (guarded against an out-of-range window map), split
    // into nz consecutive chunks
    const int tlo = max(sm.glo, 0), thi = min(sm.ghi, a.G);
    const int chunk = (thi - tlo + nz - 1) / nz;
    const int glo = tlo + bz * chunk, ghi = min(thi, glo + chunk);
    const bool use_stage = a.tmaps != nullptr && stg != nullptr;
    if (use_stage && warp == kPlanWarp && ghi > glo) {
        // the tensor maps were written to global memory by a host copy: the
        // issuing thread orders the tensor-map proxy's reads after it
        if (lane == 0)
            for (int k = 0; k < a.V; ++k)
                asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;"
                             ::"l"((uint64_t)(static_cast<const char*>(a.tmaps) + (size_t)k * 128))
                             : "memory");
        __syncwarp();
        stage_plan(a, sm, stg, tx0, ty0, glo, 0, 0, lane);
    }
    // the set-up of the first two pairs; each later pair's comes from the
    // planning warp two pairs ahead, after the barrier of the pair between
    if (warp == kPlanWarp && ghi > glo) {
        stage_setup(a, sm, tx0, ty0, glo, 0, 0, lane);
        const int g1 = a.V > 1 ? glo : glo + 1, k1 = a.V > 1 ? 1 : 0;
        if (g1 < ghi) stage_setup(a, sm, tx0, ty0, g1, k1, 1, lane);
    }
    __syncthreads();

    // census role (warps 0-6): column 8 * warp + lane % 8, rows
    // CH * (lane / 8) .. + CH - 1; warp 7 has none
    const int pc = warp * 8 + (lane & 7);
    const int pr0 = (lane >> 3) * CH;
    const bool cact = warp < kCensusWarps;
    // sampling role: sample rows [rs, re), sample columns lane and 32 + lane
    const int rs = row_start(warp), re = row_start(warp + 1);
    const float wm1 = (float)(W - 1), hm1 = (float)(H - 1);
    // tile-relative sample row of the image's last row: rows past it are read
    // from it (computing them anew would round differently from the row that
    // was stepped there, and break the exact ties the clamped reading makes)
    const int jlast = H - 1 - (ty0 - 3);
    // Windows differ across the tile (a per-pixel range of D planes), so a
    // warp skips a plane its rows do not need.  Sample row j feeds the census
    // of pixel rows j - 6 .. j (NCC: j - 5 .. j - 1, a subset) and the centre
    // bit of pixel row j - 3; the census chunk needs the planes of its own
    // pixels.  Only work is skipped, never a barrier, and the flags are
    // uniform across the warp.  A skipped sample row keeps an older plane's
    // values: it can only feed pixels whose windows exclude this plane, and
    // their results are not stored.
    int splo = a.G, sphi = 0;
    for (int r = max(rs - 6, 0); r <= min(re - 1, PH - 1); ++r) {
        splo = min(splo, sm.rlo[r]);
        sphi = max(sphi, sm.rhi[r]);
    }
    int cplo = a.G, cphi = 0;
    if (cact) {
        for (int r = 0; r < CH; ++r) {
            const int v = sm.lo[pr0 + r][pc];
            if (v != (1 << 30)) {
                cplo = min(cplo, v);
                cphi = max(cphi, v + a.D);
            }
        }
    }
    cplo = __reduce_min_sync(0xFFFFFFFFu, cplo);
    cphi = __reduce_max_sync(0xFFFFFFFFu, cphi);
    // near-tie bits of the census words that count (a pixel on the left /
    // right image edge leaves out its ties with itself)
    const uint32_t keep1 = tx0 + pc == 0 ? big_bits(1) & ~kSelfLeft : big_bits(1);
    const uint32_t keep2 = tx0 + pc == W - 1 ? big_bits(2) & ~kSelfRight : big_bits(2);

    int buf = 0;
    for (int g = glo; g < ghi; ++g) {
        uint32_t slr[CH];
#pragma unroll
        for (int r = 0; r < CH; ++r) slr[r] = 0;
        const bool do_sample = g >= splo && g < sphi;
        const bool do_cost = cact && g >= cplo && g < cphi;
        for (int k = 0; k < a.V; ++k) {
            // ---------------------------------------------------------- staging of the next pair
            if (use_stage && warp == kPlanWarp) {
                const int gn = k + 1 < a.V ? g : g + 1, kn = k + 1 < a.V ? k + 1 : 0;
                if (gn < ghi) stage_plan(a, sm, stg, tx0, ty0, gn, kn, buf ^ 1, lane);
            }
            const bool staged = use_stage && sm.stg_ok[buf];
            // every issued copy completes before the barrier below: the planning
            // warp waits for it even when it samples nothing of this plane (a
            // plane in a gap between the tile's windows is needed by no warp)
            bool ready = false;
            if (staged && (do_sample || warp == kPlanWarp)) {
                ready = stage_wait(&sm.mbar[buf], (phase >> buf) & 1u, a.stage_test ? (1LL << 21) : (1LL << 31));
                if (!ready && lane == 0) {
                    if (a.err) atomicOr(a.err, 1);
                    sm.stg_dead = 1;
                }
            }
            // ---------------------------------------------------------- sampling
            if (do_sample) {
                const uint8_t* sp = ready ? stg + buf * kStageBX * kStageBY : nullptr;
                const int sx0 = ready ? sm.stg_x0[buf] : -(1 << 20), sy0 = ready ? sm.stg_y0[buf] : -(1 << 20);
                const uint8_t* img = a.views.img[k];
                if (!NCC && lane < 18)
                    sm.hdf[buf][lane] = __ldg(a.htab + ((size_t)(FM_IN(g, a.G, 0x108) ? g : 0) * a.V + k) * 18 + lane);
                // numerators and denominator of the lane's two columns, as
                // pairs: column terms + the row term of the warp's first row
                auto start = [&](int c) {
                    const float4 x = sm.xt[buf][c][lane];
                    const float2 y = sm.yt[buf][warp][c];
                    return to_grid2(df_add2(df2{make_float2(x.x, x.y), make_float2(x.z, x.w)}, df{y.x, y.y}));
                };
                auto step = [&](int c) {
                    const float2 t = sm.st[buf][c];
                    return df2{f2(t.x), f2(t.y)};
                };
                df2 U = start(0), Vn = start(1), Dn = start(2);
                const df2 S1 = step(0), S4 = step(1), S7 = step(2);
                float(*vrow)[SW] = sm.val[buf];
                uint32_t rk_lo = 0u, rk_hi = 0u;
                // the row loop in two variants, chosen once per (plane, view):
                // every sample 2 px inside the image with its taps in the staged
                // box (no clamping, no box test), or taps from the staged box
                // where it holds them and from global memory elsewhere
                auto rows = [&](auto inner_tag) {
                constexpr bool IN = decltype(inner_tag)::value;
                // not unrolled: measured faster than unrolling by 2, 3 or 4
#pragma unroll 1
                for (int jj = 0; jj < kMaxRows; ++jj) {
                    const int j = rs + jj;
                    if (j >= re) break;
                    const int Y = ty0 - 3 + j;
                    // rows below the image repeat its last row: the census and
                    // NCC read that row for them (the same values bit for bit,
                    // as the clamped reading makes them equal)
                    if (Y > H - 1) break;
                    if (jj > 0 && Y >= 1 && Y <= H - 1) {
                        U = grid_add2(U, S1); Vn = grid_add2(Vn, S4); Dn = grid_add2(Dn, S7);
                    }
                    bool ok0 = false, ok1 = false;
                    const bool centre_row = j >= 3 && j < 3 + PH;
                    float f0, f1;
                    bool pl0, pl1;
                    if constexpr (IN) {
                        const float2 fv = taps2_staged(sp, sx0, sy0, sample_pos2_in(U, Vn, Dn), pl0, pl1);
                        f0 = fv.x;
                        f1 = fv.y;
                        ok0 = ok1 = true;
                    } else {
                        const SPos2 q = sample_pos2(wm1, hm1, U, Vn, Dn, ok0, ok1);
                        const SPos p0{q.iu0, q.iv0, q.su0, q.sv0, q.a.x, q.b.x};
                        const SPos p1{q.iu1, q.iv1, q.su1, q.sv1, q.a.y, q.b.y};
                        // a row whose taps all lie in the box (the usual case)
                        // takes one straight shared-memory path; without a box
                        // (sp null, origin far away) every tap reads global memory
                        const bool b0 = in_box(sx0, sy0, p0), b1 = in_box(sx0, sy0, p1);
                        if (__all_sync(0xFFFFFFFFu, b0 && b1)) {
                            const float2 fv = taps2_staged(sp, sx0, sy0, q, pl0, pl1);
                            f0 = fv.x;
                            f1 = fv.y;
                        } else {
                            f0 = b0 ? taps_staged(sp, sx0, sy0, p0, pl0) : taps_global(img, a.pitch, W, H, p0, pl0);
                            f1 = b1 ? taps_staged(sp, sx0, sy0, p1, pl1) : taps_global(img, a.pitch, W, H, p1, pl1);
                        }
                    }
                    if (FM_IN(j, SH, 0x103)) {
                        vrow[j][lane] = f0;
                        vrow[j][32 + lane] = f1;
                    }
                    if constexpr (!NCC) {
                        // risky samples: not a plateau but within 2^-13 of an
                        // integer; per pixel column, whether its 9 window columns
                        // hold one in this row (bit jj of the warp's byte)
                        const bool rk0 = !pl0 && fabsf(__fsub_rn(f0, rintf(f0))) < kRiskyBound;
                        const bool rk1 = !pl1 && fabsf(__fsub_rn(f1, rintf(f1))) < kRiskyBound;
                        const uint32_t q0 = __ballot_sync(0xFFFFFFFFu, rk0), q1 = __ballot_sync(0xFFFFFFFFu, rk1);
                        if (lane == 0 && FM_IN(j, SH, 0x103)) {
                            sm.rkb[buf][j][0] = q0;
                            sm.rkb[buf][j][1] = q1;
                        }
                        if (q0 | q1) {
                            const uint64_t M = ((uint64_t)q1 << 32) | q0;
                            uint64_t t = M | (M >> 1);
                            t |= t >> 2;
                            t |= t >> 4;
                            t |= M >> 8;
                            rk_lo |= (uint32_t)((t >> lane) & 1u) << jj;
                            rk_hi |= (uint32_t)((t >> (lane + 32)) & 1u) << jj;
                        }
                    }
                    if (centre_row) {
                        // every sample of an interior pair lies on the image
                        const uint32_t m0 = IN ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, ok0);
                        const uint32_t m1 = IN ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, ok1);
                        if (lane == 0) {
                            sm.okm[buf][j - 3][0] = (m0 >> 4) | (m1 << 28);
                            sm.okm[buf][j - 3][1] = m1 >> 4;
                        }
                    }
                }
                };
                if (sp && sm.stg_in[buf]) rows(std::true_type{});
                else rows(std::false_type{});
                if constexpr (!NCC) {
                    sm.rkcol[buf][warp][lane] = (uint8_t)rk_lo;
                    sm.rkcol[buf][warp][32 + lane] = (uint8_t)rk_hi;
                }
                // debug capture: this warp's sample rows that are pixel rows the
                // tile stores (each lane its own two columns, read back from
                // where it wrote them)
                if (DBG && a.dbg_warp && g == a.dbg_g && k == a.dbg_k) {
                    for (int j = rs; j < re; ++j) {
                        const int Y = ty0 - 3 + j;
                        if (j < 3 || j >= 3 + PH || Y > H - 1 || j - 3 < sm.rskip) continue;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int col = lane + 32 * h, X = tx0 - 4 + col;
                            if (col >= 4 && col < 4 + PW && X < W) a.dbg_warp[(size_t)Y * W + X] = vrow[j][col];
                        }
                    }
                }
            }
            if (staged) phase ^= 1u << buf;
            __syncthreads();
            // ---------------------------------------------------------- NCC 5x5
            if constexpr (NCC) {
                if (do_cost) {
                    // window of output row r: sample rows pr0 + r + 1 .. + 5,
                    // columns pc + 2 .. pc + 6; the last five rows are kept in
                    // registers (a ring indexed by the unrolled row)
                    const float* bp = &sm.val[buf][0][pc + 2];
                    const float* ap = &sm.ncc.refv[pr0 + 1][pc + 2];
                    float rb[5][5], ra[5][5];
                    const int sh = a.views.side[k] < 0 ? 0 : 16;
#pragma unroll
                    for (int jr = 0; jr < CH + 4; ++jr) {
                        const bool rok = FM_IN(min(pr0 + 1 + jr, jlast), SH, 0x109) &&
                                         FM_IN(pr0 + 1 + jr, SH, 0x109) && FM_IN(pc + 6, SW, 0x109);
#pragma unroll
                        for (int c = 0; c < 5; ++c) {
                            rb[jr % 5][c] = rok ? bp[min(pr0 + 1 + jr, jlast) * SW + c] : 0.0f;
                            ra[jr % 5][c] = rok ? ap[jr * SW + c] : 0.0f;
                        }
                        if (jr >= 4) {
                            const int r = jr - 4;
                            const int2 rs2 = sm.ncc.refs[pr0 + r][pc];
                            // mean of b, then the deviations: sum (b - mb)^2 and
                            // 25 cov = sum (25 a - sum a)(b - mb) (integer weights)
                            float sb = 0.0f;
#pragma unroll
                            for (int i = 0; i < 5; ++i)
#pragma unroll
                                for (int c = 0; c < 5; ++c) sb = __fadd_rn(sb, rb[i][c]);
                            const float mb = __fdiv_rn(sb, 25.0f);
                            const float nsa = (float)(-rs2.x);
                            float vb = 0.0f, cv = 0.0f;
#pragma unroll
                            for (int i = 0; i < 5; ++i)
#pragma unroll
                                for (int c = 0; c < 5; ++c) {
                                    const float e = __fsub_rn(rb[i][c], mb);
                                    vb = __fmaf_rn(e, e, vb);
                                    cv = __fmaf_rn(__fmaf_rn(25.0f, ra[i][c], nsa), e, cv);
                                }
                            uint32_t cost = 255u;
                            if (rs2.y > 0 && vb > 0.0f && cv > 0.0f) {
                                // ncc = cov / sqrt(va vb) = cv / (5 sqrt(25 va' vb)), 25 va' = refs.y
                                const float ncc = __fdiv_rn(cv, __fmul_rn(5.0f, __fsqrt_rn(__fmul_rn((float)rs2.y, vb))));
                                const float cf = __fmul_rn(255.0f, __fsub_rn(1.0f, ncc));
                                cost = (uint32_t)min(max((int)floorf(__fadd_rn(cf, 0.5f)), 0), 255);
                            }
                            const bool ok = (sm.okm[buf][pr0 + r][pc >> 5] >> (pc & 31)) & 1u;
                            if (!ok) cost = 255u;
                            slr[r] += cost << sh;
                        }
                    }
                }
            } else
            // ---------------------------------------------------------- census
            if (do_cost) {
                const float(*vt)[SW] = sm.val[buf];
                const float* base = &vt[0][pc];
                const int jl = jlast - pr0;
                // -2^15 V(p) of each pixel, twice: columns c and c + 1 of a
                // window row go through one packed fused multiply-add (each
                // half rounded as the scalar one)
                const float2 S2 = make_float2(kCensusScale, kCensusScale);
                float2 ncs[CH];
                uint32_t w[CH][4];
#pragma unroll
                for (int r = 0; r < CH; ++r) {
                    const float c = __fmul_rn(-kCensusScale, base[(pr0 + min(r + 3, jl)) * SW + 4]);
                    ncs[r] = make_float2(c, c);
#pragma unroll
                    for (int q = 0; q < 4; ++q) w[r][q] = 0u;
                }
#pragma unroll
                for (int jr = 0; jr < CH + 6; ++jr) {
                    float2 wv2[4];
                    const float* rowp = base + (pr0 + min(jr, jl)) * SW;
                    const bool rok = FM_IN(pr0 + min(jr, jl), SH, 0x104) && FM_IN(pc + 8, SW, 0x104);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        wv2[i] = rok ? make_float2(rowp[2 * i], rowp[2 * i + 1]) : make_float2(0.0f, 0.0f);
                    const float wv8 = rok ? rowp[8] : 0.0f;
#pragma unroll
                    for (int r = 0; r < CH; ++r) {
                        const int dy = jr - r;
                        if (dy < 0 || dy > 6) continue;
                        // 2^15 (V(q) - V(p)): sign = [V(q) < V(p)], bit 30 = the
                        // difference reaches 2^-14
                        float x[9];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float2 x2 = __ffma2_rn(wv2[i], S2, ncs[r]);
                            x[2 * i] = x2.x;
                            x[2 * i + 1] = x2.y;
                        }
                        x[8] = __fmaf_rn(wv8, kCensusScale, ncs[r].x);
#pragma unroll
                        for (int c = 0; c < 9; ++c) {
                            const int kb = dy * 9 + c;
                            if (kb == 31) continue;
                            w[r][cword(kb)] = __funnelshift_l(__float_as_uint(x[c]), w[r][cword(kb)], 2);
                        }
                    }
                }
                const int sh = a.views.side[k] < 0 ? 0 : 16;
                uint32_t fmask = 0u;
#pragma unroll
                for (int r = 0; r < CH; ++r) {
                    const uint4 rf = FM_IN((pr0 + r) * PW + pc, PH * PW, 0x105) ? sm.refl[pr0 + r][pc]
                                                                                 : make_uint4(0, 0, 0, 0);
                    int hcost = __popc((w[r][0] ^ rf.x) & SIGN_BITS) + __popc((w[r][1] ^ rf.y) & SIGN_BITS) +
                                __popc((w[r][2] ^ rf.z) & SIGN_BITS) + __popc((w[r][3] ^ rf.w) & SIGN_BITS);
                    uint32_t k0 = big_bits(0), k1 = keep1, k2 = keep2, k3 = big_bits(3);
                    // a first chunk row on the image's top row, a last one on its
                    // bottom row (always chunk row CH - 1, see the tile origin)
                    const bool eL = tx0 + pc == 0, eR = tx0 + pc == W - 1;
                    if (r == 0 && ty0 + pr0 == 0) {
                        k0 &= ~(eL ? self_mask(0, true, false, true, false)
                                   : (eR ? self_mask(0, false, true, true, false) : self_mask(0, false, false, true, false)));
                        k1 &= ~(eL ? self_mask(1, true, false, true, false)
                                   : (eR ? self_mask(1, false, true, true, false) : self_mask(1, false, false, true, false)));
                    }
                    if (r == CH - 1 && ty0 + pr0 + CH - 1 == H - 1) {
                        k2 &= ~(eL ? self_mask(2, true, false, false, true)
                                   : (eR ? self_mask(2, false, true, false, true) : self_mask(2, false, false, false, true)));
                        k3 &= ~(eL ? self_mask(3, true, false, false, true)
                                   : (eR ? self_mask(3, false, true, false, true) : self_mask(3, false, false, false, true)));
                    }
                    const uint32_t near = (~w[r][0] & k0) | (~w[r][1] & k1) | (~w[r][2] & k2) | (~w[r][3] & k3);
                    const bool ok = (sm.okm[buf][pr0 + r][pc >> 5] >> (pc & 31)) & 1u;
                    if (!ok) hcost = kCensusMax;
                    fmask |= (ok && near) ? (1u << r) : 0u;
                    slr[r] += (uint32_t)hcost << sh;
                }
                // near ties of pixels inside the image.  A pixel whose centre is an
                // integer and whose window holds no risky sample has only plateau
                // ties: its FP32 census is exact already
                {
                    const int m = tx0 + pc < W ? jlast - 3 - pr0 : -1;   // last chunk row inside the image
                    fmask &= m >= CH - 1 ? 0xFFFFFFFFu : (m < 0 ? 0u : (2u << m) - 1u);
                    const int r0 = sm.rskip - pr0;                        // first chunk row this tile stores
                    fmask &= r0 <= 0 ? 0xFFFFFFFFu : (r0 >= CH ? 0u : ~((1u << r0) - 1u));
                }
                if (fmask) {
                    uint64_t rows = 0;
#pragma unroll
                    for (int sw = 0; sw < NWARP; ++sw) rows |= (uint64_t)sm.rkcol[buf][sw][pc] << row_start(sw);
                    // rows past jlast were not sampled: they repeat row jlast
                    if (jlast < 63 && ((rows >> jlast) & 1u)) rows |= ~0ull << jlast;
                    const uint32_t rr = (uint32_t)(rows >> pr0);
                    uint32_t f = fmask;
                    while (f) {
                        const int r = __ffs(f) - 1;
                        f &= f - 1u;
                        const float vp = vt[min(pr0 + r + 3, jlast)][pc + 4];
                        if (vp == rintf(vp) && !((rr >> r) & 0x7Fu)) fmask &= ~(1u << r);
                    }
                }
                if (__any_sync(0xFFFFFFFFu, fmask != 0u)) {
                    int corr[CH];
                    fix_ties(a, sm, buf, k, tx0, ty0, pr0, pc, jlast, fmask, lane, corr);
#pragma unroll
                    for (int r = 0; r < CH; ++r) slr[r] += (uint32_t)(corr[r] * (1 << sh));
                }
            }
            // the planning warp has no census: the set-up of the pair two
            // ahead, into the slot this pair's sampling has finished with
            if (warp == kPlanWarp) {
                int g2 = g, k2 = k + 2;
                while (k2 >= a.V) { k2 -= a.V; ++g2; }
                if (g2 < ghi) stage_setup(a, sm, tx0, ty0, g2, k2, buf, lane);
            }
            buf ^= 1;
        }
        // -------------------------------------------------------------- store
        if (do_cost && tx0 + pc < W) {
            // the chunk's pixels are W * pstride elements apart, row by row
            size_t roff = ((size_t)(ty0 + pr0) * W + tx0 + pc) * a.pstride;
            const size_t rstride = (size_t)W * a.pstride;
#pragma unroll
            for (int r = 0; r < CH; ++r) {
                const int py = ty0 + pr0 + r;
                const int s = g - sm.lo[pr0 + r][pc];
                if (py < H && pr0 + r >= sm.rskip && s >= 0 && s < a.D) {
                    const uint32_t sl = slr[r] & 0xFFFFu, sr = slr[r] >> 16;
                    uint32_t vl = 0xFFFFFFFFu, vr = 0xFFFFFFFFu;
                    // (x * ceil(2^32 / n)) >> 32 == x / n exactly for x < 2^16, n <= 16
                    if (a.nL > 0) vl = (uint32_t)(((uint64_t)(sl * a.nmax + (a.nL >> 1)) * a.mL) >> 32);
                    if (a.nR > 0) vr = (uint32_t)(((uint64_t)(sr * a.nmax + (a.nR >> 1)) * a.mR) >> 32);
                    const size_t e = roff + (size_t)(s >> a.bshift) * a.bstride + (s & ((1 << a.bshift) - 1));
                    if (FM_IN(e, (size_t)W * H * a.Ds, 0x106)) a.S[e] = (uint16_t)min(vl, vr);
                }
                roff += rstride;
            }
        }
    }
}

template <bool NCC>
__global__ void __launch_bounds__(THREADS, 2) cost_kernel(const __grid_constant__ CostArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemCost& sm = *reinterpret_cast<SmemCost*>(smraw);
    // the arguments in shared memory, as the batched form keeps them (the
    // tile loop then has the registers for 64-bit row offsets)
    __shared__ CostArgs sa;
    {
        const int* src = reinterpret_cast<const int*>(&a);
        int* dst = reinterpret_cast<int*>(&sa);
        for (int i = threadIdx.x; i < (int)(sizeof(CostArgs) / sizeof(int)); i += THREADS) dst[i] = src[i];
    }
    stage_init(sm);
    uint32_t phase = 0;
    cost_tile<NCC, false>(sa, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, sm, nullptr, phase);
}

// Batched form: work items (frame, tile x, tile y, chunk | chunks << 16) of
// any number of frames.  With a counter the CTAs are persistent and pull items
// from it; without one, CTA i runs item i alone (short-lived CTAs, so that a
// higher-priority stream can take SMs over at CTA granularity).  The frame's
// arguments are staged in shared memory for the item.  DBG: the capture of a
// chosen pair's warped tile (dbg_warp) is compiled in.
template <bool NCC, bool DBG>
__global__ void __launch_bounds__(THREADS, 2)
cost_batch_kernel(const CostArgs* __restrict__ args, const int4* __restrict__ items, int n_items, int* counter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemCost& sm = *reinterpret_cast<SmemCost*>(smraw);
    __shared__ CostArgs sa;
    __shared__ int s_item;
    // the staging slots follow SmemCost, 128-byte aligned in the shared window
    const uint32_t base = smem_u32(smraw);
    uint8_t* stg = smraw + (((base + (uint32_t)sizeof(SmemCost) + 127u) & ~127u) - base);
    stage_init(sm);
    uint32_t phase = 0;
    int it = blockIdx.x;
    for (;;) {
        if (counter) {
            if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
            __syncthreads();
            it = s_item;
        }
        if (it >= n_items) break;
        const int4 w = items[it];
        {
            const int* src = reinterpret_cast<const int*>(args + w.x);
            int* dst = reinterpret_cast<int*>(&sa);
            for (int i = threadIdx.x; i < (int)(sizeof(CostArgs) / sizeof(int)); i += THREADS) dst[i] = src[i];
        }
        __syncthreads();
        cost_tile<NCC, DBG>(sa, w.y, w.z, w.w & 0xFFFF, w.w >> 16, sm, stg, phase);
        __syncthreads();
        if (!counter) break;
    }
}

}  // namespace

int cost_tiles_x(int W) { return (W + PW - 1) / PW; }
FM_CHECK_TAKE(check_take_cost)
int cost_tiles_y(int H) { return (H + PH - 1) / PH; }

namespace {
// SmemCost, alignment slack and the two staging slots
constexpr int kBatchSmem = (int)sizeof(SmemCost) + 128 + 2 * kStageBX * kStageBY;
// the shared-memory opt-in is a per-device function attribute
void cost_smem_optin()
{
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    const int smem = (int)sizeof(SmemCost);
    cudaFuncSetAttribute(cost_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(cost_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(cost_batch_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    cudaFuncSetAttribute(cost_batch_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    cudaFuncSetAttribute(cost_batch_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    cudaFuncSetAttribute(cost_batch_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    done[dev] = true;
}
}  // namespace

void launch_cost(const CostArgs& a, cudaStream_t st)
{
    cost_smem_optin();
    dim3 grid((a.W + PW - 1) / PW, (a.H + PH - 1) / PH, 1);
    // enough CTAs for about three waves of two CTAs per SM on 148 SMs
    const int tiles = (int)(grid.x * grid.y);
    grid.z = (unsigned)max(1, min((3 * 2 * 148 + tiles - 1) / tiles, (a.D + 7) / 8));
    if (a.cost) cost_kernel<true><<<grid, THREADS, sizeof(SmemCost), st>>>(a);
    else cost_kernel<false><<<grid, THREADS, sizeof(SmemCost), st>>>(a);
    count_launch();
}

void launch_cost_batch(const CostArgs* args, const int4* items, int n_items, int* counter, int ctas, bool ncc,
                       bool dbg, cudaStream_t st)
{
    cost_smem_optin();
    if (n_items <= 0) return;
    auto kern = ncc ? (dbg ? cost_batch_kernel<true, true> : cost_batch_kernel<true, false>)
                    : (dbg ? cost_batch_kernel<false, true> : cost_batch_kernel<false, false>);
    if (ctas > 0) {
        cudaMemsetAsync(counter, 0, sizeof(int), st);
        kern<<<ctas, THREADS, kBatchSmem, st>>>(args, items, n_items, counter);
    } else {
        kern<<<n_items, THREADS, kBatchSmem, st>>>(args, items, n_items, nullptr);
    }
    count_launch();
}

// ---------------------------------------------------------------- level tables
namespace {
__global__ void prep_level_kernel(const ViewGeom vg, const LevelPlanes lp, float* htab, float* delta)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lp.G * lp.V) return;
    int g = i / lp.V, k = i % lp.V;
    double rho = lp.rho0 + (double)g * lp.drho;
    float* o = htab + (size_t)i * 18;
    double Hm[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Hm[3 * r + c] = vg.A[k][3 * r + c] - rho * vg.e[k][r] * vg.c[k][c];
    // the homography is defined up to scale: make the homogeneous coordinate
    // 1 at the image centre (keeps |N|, |D| small for the exact-grid steps);
    // a centre behind the camera keeps its sign, so the w > 0 test is unchanged
    const double wc = Hm[6] * lp.xc + Hm[7] * lp.yc + Hm[8];
    const double sc = (wc != 0.0 && isfinite(wc)) ? 1.0 / fabs(wc) : 1.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double h = Hm[3 * r + c] * sc;
            float hi = (float)h;
            o[3 * r + c] = hi;
            o[9 + 3 * r + c] = (float)(h - (double)hi);
        }
    if (k == 0) delta[g] = (float)(1.0 / rho);
}
}  // namespace

void launch_prep_level(const ViewGeom& vg, const LevelPlanes& lp, float* htab, float* delta,
                       cudaStream_t st)
{
    int n = lp.G * lp.V;
    prep_level_kernel<<<(n + 127) / 128, 128, 0, st>>>(vg, lp, htab, delta);
    count_launch();
}

}  // namespace fm
