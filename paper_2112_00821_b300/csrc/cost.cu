// Plane-sweep census cost volume (Alg. 1 of FaSS-MVS) for sm_103a.
//
// A CTA of 8 warps owns a 56 x 52 tile of reference pixels and walks every
// plane its windows need, one (plane, view) pair per iteration:
//   1. sampling: the 64 x 58 warped sample tile (tile + 9x7 census halo) is
//      produced cooperatively -- each warp owns 7 or 8 sample rows, each
//      lane two sample columns (coalesced
//      neighbour-image reads), the homography is stepped down the column in
//      double-float arithmetic; samples are stored as FP16 pairs (V(x),
//      V(x+1)) so the census can load two at a time;
//   2. one __syncthreads (the sample tile is double-buffered);
//   3. census: warp w < 7 takes columns 8w .. 8w + 7 of the tile, lane l
//      column 8w + l % 8 and rows 13 (l / 8) .. + 12 (every lane of the seven
//      warps busy; rows 72 words apart so the four row chunks fall in
//      different shared-memory banks); for every
//      window row, five packed FP16 saturating subtractions give ten
//      comparison bits [V(q) < V(p)] which five packed FMAs add, with
//      power-of-two weights, into four FP16x2 accumulators (10 bits per half,
//      biased by 1024 so the half's bit pattern holds the integer); the XOR
//      with the reference census (pre-arranged in the same layout) and four
//      popcounts give the Hamming distance; left / right sums accumulate in
//      registers over the views and the plane's costs are stored after the
//      last view.
// Sampling reading (shared with the oracle): 1/256-pixel fixed-point
// positions floor(256 u), exact integer bilinear blend with 8-bit weights,
// value kept at 1/16 grey level.  Values lie in [0, 4080]; shifted by -2040
// they are exact FP16 integers, and the FP16 difference of two of them keeps
// its sign and its >= 1 test, so the census comparisons are exact.
#include <cuda_fp16.h>

#include <type_traits>

#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int PW = 56, PH = 52;          // pixel tile
constexpr int SW = 72, SH = PH + 6;      // sample tile rows: 64 samples (PW + 8) in a 72-word stride
constexpr int NWARP = 8, THREADS = 256;
constexpr int CH = 13;                   // pixel rows per census chunk (PH / 4)
constexpr int kCensusWarps = PW / 8;     // 7 warps x (8 columns x 4 chunks of 13 rows)
constexpr int kPlanWarp = NWARP - 1;     // plans and issues the staging copies
// first sample row of warp w's share (7 or 8 rows each)
__host__ __device__ constexpr int row_start(int w) { return (SH * w) / NWARP; }
constexpr int kMaxRows = 8;              // the largest share
static_assert(row_start(NWARP) - row_start(NWARP - 1) <= kMaxRows, "row shares");
constexpr int PMAX = 1 << 24;
constexpr float MAGIC = 12582912.0f;     // 1.5 * 2^23: adding it leaves an integer in the mantissa
constexpr int MAGIC_BITS = 0x4B400000;
constexpr uint32_t LAYOUT_MASK = 0x03FF03FFu;

struct SmemCost {
    uint64_t mbar[2];                    // staging: completion of the tensor copy into slot 0 / 1
    int stg_x0[2], stg_y0[2], stg_ok[2]; // staging: box origin in the view image, and whether it was issued
    int stg_dead;                        // a staged copy missed its bound: no further staging in this CTA
    uint32_t pair[2][SH][SW];            // census: FP16x2 (V(x) - 2040, V(x+1) - 2040); NCC: u16x2 (V(x), V(x+1))
    uint32_t okm[2][PH][2];              // centre-in-image bit per pixel column
    union {
        uint4 refl[PH][PW];              // census: reference census in the accumulator layout
        struct {
            uint32_t refp[SH][SW];       // NCC: reference values (a(x), a(x+1)) on the sample grid
            int2 refs[PH][PW];           // NCC: (sum a, 25 sum a^2 - (sum a)^2) of each 5x5 window
        } ncc;
    };
    int32_t lo[PH][PW];
    int32_t rlo[PH], rhi[PH];            // per pixel row: planes its windows need, [rlo, rhi)
    int glo, ghi;
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

// Values whose high word lies on the 2^-10 grid with magnitude below 2^14
// add exactly in FP32, so stepping down a column costs two additions: the
// homography is scaled (prep_level_kernel) so that |N|, |D| stay below 2^14
// over and well around the image, and the step's high words are on the grid.
constexpr float GRID_MAGIC = 12288.0f;   // 1.5 * 2^13: rounds |x| < 2^12 to the 2^-10 grid
__device__ __forceinline__ df to_grid(df a)
{
    float h = __fsub_rn(__fadd_rn(a.hi, GRID_MAGIC), GRID_MAGIC);
    return {h, __fadd_rn(a.lo, __fsub_rn(a.hi, h))};
}
__device__ __forceinline__ df grid_add(df a, df b) { return {__fadd_rn(a.hi, b.hi), __fadd_rn(a.lo, b.lo)}; }
// The denominator D is carried divided by 256 (exact: a power of two), which
// puts its high words on the 2^-18 grid with |D / 256| < 2^4 and lets the
// reciprocal give 256 / D directly.
constexpr float DGRID_MAGIC = 48.0f;     // 1.5 * 2^5: rounds |x| < 2^4 to the 2^-18 grid
__device__ __forceinline__ df to_dgrid(df a)
{
    float h = __fsub_rn(__fadd_rn(a.hi, DGRID_MAGIC), DGRID_MAGIC);
    return {h, __fadd_rn(a.lo, __fsub_rn(a.hi, h))};
}
__device__ __forceinline__ df df_scale(df a, float s) { return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)}; }

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

// floor(256 N / D) for D > 0, given Dn = D / 256 and r ~ 256 / D, for
// |N / D| < 16000: q = 256 N / D to a few ulps, the double-float residual
// N - (q / 256) D = N - q Dn gives the correction, and the floors come from
// adding 1.5 * 2^23 with round-down.  The words of N and D are split on a
// grid, so the low words are not small: q and r are formed from the summed
// words.
__device__ __forceinline__ int fix_pos(df N, df Dn, float r)
{
    float q = __fmul_rn(__fadd_rn(N.hi, N.lo), r);
    float e1 = __fmaf_rn(-q, Dn.hi, N.hi);
    float e2 = __fmaf_rn(-q, Dn.lo, N.lo);
    float corr = __fmul_rn(__fadd_rn(e1, e2), r);
    float a = fminf(fmaxf(q, -4194000.0f), 4194000.0f);
    float t1 = __fadd_rd(a, MAGIC);
    float fa = __fsub_rn(t1, MAGIC);
    float rem = __fadd_rn(corr, __fsub_rn(a, fa));
    float t2 = __fadd_rd(rem, MAGIC);
    return (__float_as_int(t1) - MAGIC_BITS) + (__float_as_int(t2) - MAGIC_BITS);
}

// The clamped tap position of one warped sample and whether the position
// lies on the image grid.  Dn is the denominator divided by 256; its sign is
// that of the exact sum of its words (rounding keeps the sign).
struct SPos { int iu, iv, A, B; };

template <bool WANT_OK>
__device__ __forceinline__ SPos sample_pos(int W, int H, df Nu, df Nv, df Dn, bool& ok)
{
    int Pu = -PMAX, Pv = -PMAX;
    const float dsum = __fadd_rn(Dn.hi, Dn.lo);
    const bool front = dsum > 0.0f;
    if (front) {
        const float r = rcp_approx(dsum);
        Pu = fix_pos(Nu, Dn, r);
        Pv = fix_pos(Nv, Dn, r);
    }
    const int wmax = 256 * (W - 1), hmax = 256 * (H - 1);
    if (WANT_OK) ok = front && Pu >= 0 && Pu <= wmax && Pv >= 0 && Pv <= hmax;
    const int cu = min(max(Pu, 0), wmax), cv = min(max(Pv, 0), hmax);
    const int iu = min(cu >> 8, W - 2), iv = min(cv >> 8, H - 2);
    return {iu, iv, cu - 256 * iu, cv - 256 * iv};
}

// exact integer bilinear blend with 8-bit weights: V = 16 x grey level in [0, 4080]
__device__ __forceinline__ int blend(int i00, int i01, int i10, int i11, int A, int B)
{
    const int top = (i00 << 8) + A * (i01 - i00);
    const int bot = (i10 << 8) + A * (i11 - i10);
    return ((top << 8) + B * (bot - top) + 2048) >> 12;
}

// the 2x2 taps from global memory
__device__ __forceinline__ int taps_global(const uint8_t* __restrict__ img, int pitch, SPos p)
{
    const uint8_t* r0 = img + (size_t)p.iv * pitch + p.iu;
    return blend(__ldg(r0), __ldg(r0 + 1), __ldg(r0 + pitch), __ldg(r0 + pitch + 1), p.A, p.B);
}

// the 2x2 taps from the staged box whose origin is (sx0, sy0) (in_box true)
__device__ __forceinline__ int taps_staged(const uint8_t* stg, int sx0, int sy0, SPos p)
{
    const uint8_t* r0 = stg + (p.iv - sy0) * kStageBX + (p.iu - sx0);
    return blend(r0[0], r0[1], r0[kStageBX], r0[kStageBX + 1], p.A, p.B);
}

__device__ __forceinline__ bool in_box(int sx0, int sy0, SPos p)
{
    return (unsigned)(p.iu - sx0) <= (unsigned)(kStageBX - 2) && (unsigned)(p.iv - sy0) <= (unsigned)(kStageBY - 2);
}

// V - 2040 as a float (exact), ready for FP16
__device__ __forceinline__ float v16_centred(int v16) { return __int_as_float(MAGIC_BITS + v16) - (MAGIC + 2040.0f); }

// canonical 9x7 census word -> four accumulator words: window row dy, pair p
// (columns 2p, 2p+1) is packed-FMA number m = 5 dy + p, which lands in word
// m / 10 at bit m % 10 of the low (even column) / high (odd column) half
__device__ __forceinline__ uint4 to_layout(uint64_t c)
{
    uint32_t w[4];
#pragma unroll
    for (int R = 0; R < 4; ++R) {
        uint32_t v = 0x64006400u;
#pragma unroll
        for (int b = 0; b < 10; ++b) {
            const int m = 10 * R + b;
            if (m >= 35) break;
            const int dy = m / 5, p = m % 5;
            v |= (uint32_t)((c >> (dy * 9 + 2 * p)) & 1u) << b;
            if (2 * p + 1 <= 8) v |= (uint32_t)((c >> (dy * 9 + 2 * p + 1)) & 1u) << (16 + b);
        }
        w[R] = v;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ __half2 as_h2(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }
__device__ __forceinline__ uint32_t as_u32(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

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
        const float y = (float)((lane & 2) ? min(max(ty0 + 54, 0), a.H - 1) : min(max(ty0 - 3, 0), a.H - 1));
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
        int ok = 0, x0 = 0, y0 = 0;
        if (all_front && !sm.stg_dead) {
            const float wm = (float)(a.W - 1), hm = (float)(a.H - 1);
            const float ulo = fminf(fmaxf(umin, 0.0f), wm), uhi = fminf(fmaxf(umax, 0.0f), wm);
            const float vlo = fminf(fmaxf(vmin, 0.0f), hm), vhi = fminf(fmaxf(vmax, 0.0f), hm);
            x0 = max((int)floorf(ulo) - 2, 0) & ~15;
            y0 = max((int)floorf(vlo) - 2, 0);
            ok = (int)floorf(uhi) + 3 <= x0 + kStageBX - 1 && (int)floorf(vhi) + 3 <= y0 + kStageBY - 1;
        }
        sm.stg_x0[slot] = x0;
        sm.stg_y0[slot] = y0;
        sm.stg_ok[slot] = ok;
        if (ok && !a.stage_test)
            stage_issue(&sm.mbar[slot], stg + slot * kStageBX * kStageBY,
                        static_cast<const char*>(a.tmaps) + (size_t)k * 128, x0, y0);
    }
}

// One tile (bx, by) of one frame, plane chunk bz of nz, with the census (NCC
// false) or NCC 5x5 cost.  Called by the single-frame grid kernel and by the
// multi-frame kernel.  ROWSTEP: the volume stores step a 64-bit offset from
// row to row (fewer instructions; the multi-frame kernel, whose arguments sit
// in shared memory, has the registers for it, the single-frame one would
// spill).
template <bool NCC, bool ROWSTEP>
__device__ __forceinline__ void cost_tile(const CostArgs& a, int bx, int by, int bz, int nz, SmemCost& sm,
                                          uint8_t* stg, uint32_t& phase)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx0 = bx * PW, ty0 = by * PH;
    const int W = a.W, H = a.H;

    if (tid == 0) { sm.glo = a.G; sm.ghi = 0; }
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
        // 5x5 window sums
        for (int i = tid; i < SH * SW; i += THREADS) {
            const int j = i / SW, c = i % SW;
            const uint8_t* row = a.ref + (size_t)min(max(ty0 - 3 + j, 0), H - 1) * a.ref_pitch;
            const int x0 = min(max(tx0 - 4 + c, 0), W - 1), x1 = min(max(tx0 - 3 + c, 0), W - 1);
            sm.ncc.refp[j][c] = (uint32_t)__ldg(row + x0) | ((uint32_t)__ldg(row + x1) << 16);
        }
        __syncthreads();
        for (int i = tid; i < PH * PW; i += THREADS) {
            const int r = i / PW, c = i % PW;
            int sa = 0, saa = 0;
#pragma unroll
            for (int dy = 0; dy < 5; ++dy)
#pragma unroll
                for (int dx = 0; dx < 5; ++dx) {
                    const int v = (int)(sm.ncc.refp[r + 1 + dy][c + 2 + dx] & 0xFFFFu);
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
    for (int i = tid; i < 2 * SH * SW; i += THREADS) (&sm.pair[0][0][0])[i] = 0u;
    for (int i = tid; i < 2 * PH * 2; i += THREADS) (&sm.okm[0][0][0])[i] = 0u;
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
    __syncthreads();

    // census role (warps 0-6): column 8 * warp + lane % 8, rows
    // 13 * (lane / 8) .. + 12; warp 7 has none
    const int pc = warp * 8 + (lane & 7);
    const int pr0 = (lane >> 3) * CH;
    const bool cact = warp < kCensusWarps;
    // sampling role: sample rows [rs, re), sample columns lane and 32 + lane
    const int rs = row_start(warp), re = row_start(warp + 1);
    const int X0 = min(max(tx0 - 4 + lane, 0), W - 1);
    const int X1 = min(max(tx0 + 28 + lane, 0), W - 1);
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
                const int sx0 = ready ? sm.stg_x0[buf] : 0, sy0 = ready ? sm.stg_y0[buf] : 0;
                const float* h = a.htab + ((size_t)g * a.V + k) * 18;
                const uint8_t* img = a.views.img[k];
                const df h0 = load_df(h, 0), h1 = load_df(h, 1), h2 = load_df(h, 2);
                const df h3 = load_df(h, 3), h4 = load_df(h, 4), h5 = load_df(h, 5);
                const df h6 = df_scale(load_df(h, 6), 0.00390625f), h7 = df_scale(load_df(h, 7), 0.00390625f);
                const df h8 = df_scale(load_df(h, 8), 0.00390625f);     // the denominator row / 256
                const float fy = (float)min(max(ty0 - 3 + rs, 0), H - 1);
                const float fx0 = (float)X0, fx1 = (float)X1;
                const df by_u = df_add(df_mul_int(h1, fy), h2);
                const df by_v = df_add(df_mul_int(h4, fy), h5);
                const df by_d = df_add(df_mul_int(h7, fy), h8);
                df u0 = to_grid(df_add(df_mul_int(h0, fx0), by_u)), v0 = to_grid(df_add(df_mul_int(h3, fx0), by_v));
                df d0 = to_dgrid(df_add(df_mul_int(h6, fx0), by_d));
                df u1 = to_grid(df_add(df_mul_int(h0, fx1), by_u)), v1 = to_grid(df_add(df_mul_int(h3, fx1), by_v));
                df d1 = to_dgrid(df_add(df_mul_int(h6, fx1), by_d));
                const df s1 = to_grid(h1), s4 = to_grid(h4), s7 = to_dgrid(h7);
                uint32_t(*prow)[SW] = sm.pair[buf];
                // the row loop in two variants, chosen once per (plane, view):
                // taps from the staged box (global memory outside it), or from
                // global memory only
                auto rows = [&](auto staged_tag) {
                constexpr bool ST = decltype(staged_tag)::value;
                // not unrolled: measured faster than unrolling by 2, 3 or 4
#pragma unroll 1
                for (int jj = 0; jj < kMaxRows; ++jj) {
                    const int j = rs + jj;
                    if (j >= re) break;
                    const int Y = ty0 - 3 + j;
                    if (jj > 0 && Y >= 1 && Y <= H - 1) {
                        u0 = grid_add(u0, s1); v0 = grid_add(v0, s4); d0 = grid_add(d0, s7);
                        u1 = grid_add(u1, s1); v1 = grid_add(v1, s4); d1 = grid_add(d1, s7);
                    }
                    bool ok0 = false, ok1 = false;
                    const bool centre_row = j >= 3 && j < 3 + PH;
                    int i0, i1;
                    SPos p0, p1;
                    if (centre_row) {
                        p0 = sample_pos<true>(W, H, u0, v0, d0, ok0);
                        p1 = sample_pos<true>(W, H, u1, v1, d1, ok1);
                    } else {
                        p0 = sample_pos<false>(W, H, u0, v0, d0, ok0);
                        p1 = sample_pos<false>(W, H, u1, v1, d1, ok1);
                    }
                    if constexpr (ST) {
                        // a row whose taps all lie in the box (the usual case)
                        // takes one straight shared-memory path
                        const bool b0 = in_box(sx0, sy0, p0), b1 = in_box(sx0, sy0, p1);
                        if (__all_sync(0xFFFFFFFFu, b0 && b1)) {
                            i0 = taps_staged(sp, sx0, sy0, p0);
                            i1 = taps_staged(sp, sx0, sy0, p1);
                        } else {
                            i0 = b0 ? taps_staged(sp, sx0, sy0, p0) : taps_global(img, a.pitch, p0);
                            i1 = b1 ? taps_staged(sp, sx0, sy0, p1) : taps_global(img, a.pitch, p1);
                        }
                    } else {
                        i0 = taps_global(img, a.pitch, p0);
                        i1 = taps_global(img, a.pitch, p1);
                    }
                    if constexpr (NCC) {
                        int n0 = __shfl_sync(0xFFFFFFFFu, i0, (lane + 1) & 31);
                        const int t1 = __shfl_sync(0xFFFFFFFFu, i1, 0);
                        int n1 = __shfl_sync(0xFFFFFFFFu, i1, (lane + 1) & 31);
                        if (lane == 31) { n0 = t1; n1 = 0; }
                        prow[j][lane] = (uint32_t)i0 | ((uint32_t)n0 << 16);
                        prow[j][32 + lane] = (uint32_t)i1 | ((uint32_t)n1 << 16);
                    } else {
                        const float q0 = v16_centred(i0), q1 = v16_centred(i1);
                        float n0 = __shfl_sync(0xFFFFFFFFu, q0, (lane + 1) & 31);
                        const float t1 = __shfl_sync(0xFFFFFFFFu, q1, 0);
                        float n1 = __shfl_sync(0xFFFFFFFFu, q1, (lane + 1) & 31);
                        if (lane == 31) { n0 = t1; n1 = 0.0f; }
                        prow[j][lane] = as_u32(__floats2half2_rn(q0, n0));
                        prow[j][32 + lane] = as_u32(__floats2half2_rn(q1, n1));
                    }
                    if (centre_row) {
                        const uint32_t m0 = __ballot_sync(0xFFFFFFFFu, ok0);
                        const uint32_t m1 = __ballot_sync(0xFFFFFFFFu, ok1);
                        if (lane == 0) {
                            sm.okm[buf][j - 3][0] = (m0 >> 4) | (m1 << 28);
                            sm.okm[buf][j - 3][1] = m1 >> 4;
                        }
                    }
                }
                };
                if (sp) rows(std::true_type{});
                else rows(std::false_type{});
            }
            if (staged) phase ^= 1u << buf;
            __syncthreads();
            // ---------------------------------------------------------- NCC 5x5
            if constexpr (NCC) {
                if (do_cost) {
                    // window of output row r: sample rows pr0 + r + 1 .. + 5,
                    // columns pc + 2 .. pc + 6; row sums slide down the column
                    const uint32_t* bp = &sm.pair[buf][pr0 + 1][pc + 2];
                    const uint32_t* ap = &sm.ncc.refp[pr0 + 1][pc + 2];
                    int hb[5], hbb[5], hab[5];
                    int Sb = 0, Sbb = 0, Sab = 0;
                    const int sh = a.views.side[k] < 0 ? 0 : 16;
#pragma unroll
                    for (int jr = 0; jr < CH + 4; ++jr) {
                        const uint32_t w0 = bp[jr * SW], w1 = bp[jr * SW + 2], w2 = bp[jr * SW + 4];
                        const uint32_t x0 = ap[jr * SW], x1 = ap[jr * SW + 2], x2 = ap[jr * SW + 4];
                        const int b0 = w0 & 0xFFFF, b1 = w0 >> 16, b2 = w1 & 0xFFFF, b3 = w1 >> 16, b4 = w2 & 0xFFFF;
                        const int a0 = x0 & 0xFFFF, a1 = x0 >> 16, a2 = x1 & 0xFFFF, a3 = x1 >> 16, a4 = x2 & 0xFFFF;
                        const int rb = b0 + b1 + b2 + b3 + b4;
                        const int rbb = b0 * b0 + b1 * b1 + b2 * b2 + b3 * b3 + b4 * b4;
                        const int rab = a0 * b0 + a1 * b1 + a2 * b2 + a3 * b3 + a4 * b4;
                        Sb += rb;
                        Sbb += rbb;
                        Sab += rab;
                        if (jr >= 5) {
                            Sb -= hb[jr % 5];
                            Sbb -= hbb[jr % 5];
                            Sab -= hab[jr % 5];
                        }
                        hb[jr % 5] = rb;
                        hbb[jr % 5] = rbb;
                        hab[jr % 5] = rab;
                        if (jr >= 4) {
                            const int r = jr - 4;
                            const int2 rs = sm.ncc.refs[pr0 + r][pc];
                            const long long cov = 25LL * Sab - (long long)rs.x * Sb;
                            const long long vb = 25LL * Sbb - (long long)Sb * Sb;
                            uint32_t c = 255u;
                            if (rs.y > 0 && vb > 0 && cov > 0) {
                                // single precision, each step correctly rounded, in the
                                // oracle's order
                                const float fa = __int2float_rn(rs.y), fb = __ll2float_rn(vb);
                                const float ncc = __fdiv_rn(__ll2float_rn(cov), __fsqrt_rn(__fmul_rn(fa, fb)));
                                const float cf = __fmul_rn(255.0f, __fsub_rn(1.0f, ncc));
                                c = (uint32_t)min(max((int)floorf(__fadd_rn(cf, 0.5f)), 0), 255);
                            }
                            const bool ok = (sm.okm[buf][pr0 + r][pc >> 5] >> (pc & 31)) & 1u;
                            if (!ok) c = 255u;
                            slr[r] += c << sh;
                        }
                    }
                }
            } else
            // ---------------------------------------------------------- census
            if (do_cost) {
                const uint32_t* base = &sm.pair[buf][pr0][pc];
                __half2 cen[CH];
                __half2 acc[CH][4];
                const __half2 bias = __floats2half2_rn(1024.0f, 1024.0f);
#pragma unroll
                for (int r = 0; r < CH; ++r) {
                    cen[r] = __low2half2(as_h2(base[(r + 3) * SW + 4]));
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = bias;
                }
#pragma unroll
                for (int jr = 0; jr < CH + 6; ++jr) {
                    __half2 wv[5];
#pragma unroll
                    for (int p = 0; p < 5; ++p) wv[p] = as_h2(base[jr * SW + 2 * p]);
#pragma unroll
                    for (int r = 0; r < CH; ++r) {
                        const int dy = jr - r;
                        if (dy < 0 || dy > 6) continue;
#pragma unroll
                        for (int p = 0; p < 5; ++p) {
                            const int m = dy * 5 + p;
                            const float wt = (float)(1 << (m % 10));
                            const __half2 w2 = __floats2half2_rn(wt, p == 4 ? 0.0f : wt);
                            const __half2 bits = __hsub2_sat(cen[r], wv[p]);
                            acc[r][m / 10] = __hfma2(bits, w2, acc[r][m / 10]);
                        }
                    }
                }
                const int sh = a.views.side[k] < 0 ? 0 : 16;
#pragma unroll
                for (int r = 0; r < CH; ++r) {
                    const uint4 rf = sm.refl[pr0 + r][pc];
                    uint32_t hcost = __popc((as_u32(acc[r][0]) ^ rf.x) & LAYOUT_MASK) +
                                     __popc((as_u32(acc[r][1]) ^ rf.y) & LAYOUT_MASK) +
                                     __popc((as_u32(acc[r][2]) ^ rf.z) & LAYOUT_MASK) +
                                     __popc((as_u32(acc[r][3]) ^ rf.w) & LAYOUT_MASK);
                    const bool ok = (sm.okm[buf][pr0 + r][pc >> 5] >> (pc & 31)) & 1u;
                    if (!ok) hcost = kCensusMax;
                    slr[r] += hcost << sh;
                }
            }
            buf ^= 1;
        }
        // -------------------------------------------------------------- store
        if (do_cost && tx0 + pc < W) {
            // the chunk's pixels are W * pstride elements apart, row by row
            size_t roff = ROWSTEP ? ((size_t)(ty0 + pr0) * W + tx0 + pc) * a.pstride : 0;
            const size_t rstride = ROWSTEP ? (size_t)W * a.pstride : 0;
#pragma unroll
            for (int r = 0; r < CH; ++r) {
                const int py = ty0 + pr0 + r;
                const int s = g - sm.lo[pr0 + r][pc];
                if (py < H && s >= 0 && s < a.D) {
                    const uint32_t sl = slr[r] & 0xFFFFu, sr = slr[r] >> 16;
                    uint32_t vl = 0xFFFFFFFFu, vr = 0xFFFFFFFFu;
                    // (x * ceil(2^32 / n)) >> 32 == x / n exactly for x < 2^16, n <= 16
                    if (a.nL > 0) vl = (uint32_t)(((uint64_t)(sl * a.nmax + (a.nL >> 1)) * a.mL) >> 32);
                    if (a.nR > 0) vr = (uint32_t)(((uint64_t)(sr * a.nmax + (a.nR >> 1)) * a.mR) >> 32);
                    const size_t poff = ROWSTEP ? roff : ((size_t)py * W + tx0 + pc) * a.pstride;
                    a.S[poff + (size_t)(s >> a.bshift) * a.bstride + (s & ((1 << a.bshift) - 1))] =
                        (uint16_t)min(vl, vr);
                }
                roff += rstride;
            }
        }
    }
}

template <bool NCC>
__global__ void __launch_bounds__(THREADS, 2) cost_kernel(const CostArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    SmemCost& sm = *reinterpret_cast<SmemCost*>(smraw);
    stage_init(sm);
    uint32_t phase = 0;
    cost_tile<NCC, false>(a, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, sm, nullptr, phase);
}

// Batched form: work items (frame, tile x, tile y, chunk | chunks << 16) of
// any number of frames.  With a counter the CTAs are persistent and pull items
// from it; without one, CTA i runs item i alone (short-lived CTAs, so that a
// higher-priority stream can take SMs over at CTA granularity).  The frame's
// arguments are staged in shared memory for the item.
template <bool NCC>
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
        cost_tile<NCC, true>(sa, w.y, w.z, w.w & 0xFFFF, w.w >> 16, sm, stg, phase);
        __syncthreads();
        if (!counter) break;
    }
}

}  // namespace

int cost_tiles_x(int W) { return (W + PW - 1) / PW; }
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
    cudaFuncSetAttribute(cost_batch_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    cudaFuncSetAttribute(cost_batch_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
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
                       cudaStream_t st)
{
    cost_smem_optin();
    if (n_items <= 0) return;
    auto kern = ncc ? cost_batch_kernel<true> : cost_batch_kernel<false>;
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
