// Semi-global matching in two wavefront passes (Sec. 2.3 of FaSS-MVS) with the
// winner-takes-all and sub-plane refinement (Sec. 2.3.4) fused, for sm_103a.
//
// Pass A walks every image row left to right, the rows top to bottom, and
// runs the four paths whose predecessor lies to the left or in the row above:
// (1,0), (0,1), (1,1) and (-1,1).  Pass B walks the image rotated by half a
// turn -- rows bottom to top, right to left -- and runs the other four:
// (-1,0), (0,-1), (-1,-1), (1,-1).  One warp owns one row and steps its
// paths together (one batched step per column); lane l holds hypotheses
// 8l .. 8l+7 of the current pixel, two per register.  The horizontal path
// keeps its predecessor in registers.  The three paths that come from the row
// above read the predecessor's costs, minimum and winning planes from the warp
// of that row through a ring of NS columns in shared memory; the first warp of
// a block of kWaveRows rows reads them from the last warp of the block above
// through a ring in global memory.  A warp starts a column once the row above
// has published the column to its right, and publishes a column once the warp
// below has read the column NS places before it (bounded waits; a wait that
// gives up raises an error word and makes every later wait return at once).
// Blocks take tickets in launch order, so the block above always runs first
// and every wait ends.
//
// Pass A writes the sum of its four paths (T1, 16 bits per hypothesis).  Pass
// B adds its own four and T1: the whole aggregate S_bar of Eq. sgm-aggr,
// without a stored aggregate or partial sums, and takes the winner and the
// parabola in place.  DRAM traffic per voxel: S read twice, T1 written and
// read once (8 bytes), against 4 bytes for one read of S and one write of
// S_bar; the aggregate is written only for a debug capture.
//
// Every recurrence step is the one of sgm.cu (Eq. xsgm, sgm-smooth-*, the
// normalised form with windows); the sum is exact (every total stays below
// 2^16, checked on the host), so the results equal the per-direction kernels'
// bit for bit.
//
// Measured on a single frame it is latency-bound: the wavefront walks
// 2 H + W columns in sequence (a row starts two columns behind the row above)
// where a path line walks at most max(W, H), and one column step of a row
// costs about one line step per path (with every wait between rows removed,
// 2.4 us per column at 160 x 120).  At 1080p x 256 planes (four levels) it
// takes 52 ms against 5.6 ms for the per-direction kernels and the separate
// winner-takes-all, so it is the explicit form sgm_parts = -1, not the
// default.
#include <algorithm>
#include <map>
#include <mutex>

#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int R = kWaveRows;
constexpr int NS = 8;                      // shared ring columns per warp (a power of two)
constexpr int NG = kWaveRing;              // global ring columns per block boundary (at least)
// Between CTAs a fence costs about a trip to L2 and waits for the warp's
// outstanding stores, so the global flags move every KG columns (and at the
// row's end); the ring holds NG >= 4 KG columns so the producer seldom waits.
constexpr int KG = 4;
static_assert(NG >= 4 * KG, "ring shorter than the flag period allows");
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint32_t INF16 = 0x3FFFu;
constexpr uint32_t INF2 = INF16 | (INF16 << 16);
__device__ __forceinline__ uint32_t dup2(uint32_t v) { return v | (v << 16); }

// Per column a row publishes, for each of its cross-row paths, the costs of
// the lane's slots and {minimum, winning plane, the predecessor's winning
// plane}; and the column's {window start, image value}.
struct WaveSmem {
    uint4 L[R][NS][3][32];
    int4 sc[R][NS][4];
    uint16_t buf[R][4 * (kMaxSlots + 4)];  // per warp and path: the window shift
    int prog[R];                           // columns each warp has published
    int cons[R];                           // columns each warp has consumed from the row above
    int item;
};

// Flags between rows.  Within a CTA they live in shared memory, between CTAs
// in global memory; the writer stores its data, syncs its warp and then lane
// 0 stores the flag with release semantics, the reader's lane 0 loads it with
// acquire semantics and syncs its warp before reading the data.
__device__ __forceinline__ int ld_acquire_gpu(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int* p)
{
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];"
                 : "=r"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v)
{
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
}

// Bounded wait: lane 0 polls until *flag >= need and the warp gets the value
// seen.  After about a second (2^31 cycles) of polling, or once another wait
// of the launch has given up, it raises the error word and returns `need`
// (the row then finishes on whatever the buffers hold, the estimate is
// reported failed by the error word).
template <bool GLOBAL>
__device__ __forceinline__ int wait_at_least(const int* flag, int need, int* err, int lane)
{
    int v = need;
    if (lane == 0) {
        const long long t0 = clock64();
        for (unsigned it = 1;; ++it) {
            const int f = GLOBAL ? ld_acquire_gpu(flag) : ld_acquire_cta(flag);
            if (f >= need) { v = f; break; }
            if ((it & 63) == 0) {          // the error word and the clock now and then
                if (*(volatile const int*)err != 0) break;
                if (clock64() - t0 > (1LL << 31)) {
                    atomicOr(err, 2);
                    break;
                }
            }
        }
    }
    v = __shfl_sync(FULL, v, 0);
    __syncwarp();
    return v;
}

// One step of the NP path recurrences of a pass (Eq. xsgm in the normalised
// form, the penalties of Eq. sgm-smooth-* and p2-grad, windows) for the
// warp's pixel, in phases over the paths -- neighbour shuffles and
// transitions, one shift round through the warp's buffers, the new costs, NP
// independent minimum reductions -- so that the paths' dependency chains
// overlap.  Per path p: Lp the predecessor's costs (two slots per register,
// INF16 outside its window), Mp its minimum, sigma the slot shift
// lo_p - lo_pred + di, P2 the large penalty; first: the path starts here
// (L = S).  Returns the pixel's costs in L, their minimum in M and, for the
// path-gradient variant, the winning slot (lowest on ties).  The arithmetic of
// each path is that of sgm.cu's line walk, so the sums agree bit for bit.
struct PathIn {
    int D, s0, lane, variant, p1;
    uint32_t vmask[4];
};
constexpr int kBufLen = kMaxSlots + 4;     // one shift buffer per path and warp

template <int NP>
__device__ __forceinline__ void paths_step(const PathIn& q, const uint32_t (&Sv)[4], const uint32_t (&Lp)[NP][4],
                                           const uint32_t (&Mp)[NP], const bool (&first)[NP],
                                           const int (&sigma)[NP], const int (&P2)[NP], uint16_t* buf,
                                           uint32_t (&L)[NP][4], uint32_t (&M)[NP], int (&wslot)[NP])
{
    const uint32_t P1 = (uint32_t)q.p1, P1P1 = dup2(P1);
    uint32_t T[NP][4], cap[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        uint32_t left = __shfl_up_sync(FULL, Lp[p][3], 1), right = __shfl_down_sync(FULL, Lp[p][0], 1);
        if (q.lane == 0) left = INF2;
        if (q.lane == 31) right = INF2;
        cap[p] = Mp[p] + (uint32_t)max(P2[p], q.p1);
        const uint32_t cap2 = dup2(cap[p]);
        // T(s') = min(L'(s'), L'(s'-1) + P1, L'(s'+1) + P1, M' + P2), packed
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t pv = __byte_perm(j == 0 ? left : Lp[p][j - 1], Lp[p][j], 0x5432);
            const uint32_t nv = __byte_perm(Lp[p][j], j == 3 ? right : Lp[p][j + 1], 0x5432);
            T[p][j] = __vimin3_u16x2(Lp[p][j], cap2, __viaddmin_u16x2(pv, P1P1, nv + P1P1));
        }
    }
    bool shift[NP], any = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        shift[p] = !first[p] && sigma[p] != 0;     // warp-uniform
        any |= shift[p];
    }
    if (any) {
        // shift by sigma slots through the path's buffer: index k + 2 holds
        // T(k) for k in [-2, D+1]; beyond the predecessor's window the
        // transition costs M' + P2 (k = -2, D + 1 and clamped indices)
        const int D = q.D, s0 = q.s0;
        const int lastl = (D - 1) >> 3, lasti = (D - 1) & 7;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (!shift[p]) continue;
            uint16_t* bp = buf + p * kBufLen;
            uint32_t* b32 = reinterpret_cast<uint32_t*>(bp);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (s0 + 2 * j + 1 < D) b32[1 + (s0 >> 1) + j] = T[p][j];
                else if (s0 + 2 * j < D) bp[2 + s0 + 2 * j] = (uint16_t)(T[p][j] & 0xFFFFu);
            }
            const uint32_t lp0 = __shfl_sync(FULL, Lp[p][0], 0) & 0xFFFFu;
            // Lp[lasti >> 1] by selects (an indexed read would go to local memory)
            const uint32_t l01 = (lasti & 2) ? Lp[p][1] : Lp[p][0], l23 = (lasti & 2) ? Lp[p][3] : Lp[p][2];
            const uint32_t lsel = (lasti & 4) ? l23 : l01;
            const uint32_t lpw = __shfl_sync(FULL, lsel, lastl);
            const uint32_t lpD = (lasti & 1) ? (lpw >> 16) : (lpw & 0xFFFFu);
            if (q.lane == 0) {
                bp[0] = (uint16_t)cap[p];
                bp[1] = (uint16_t)min(lp0 + P1, cap[p]);
                bp[D + 2] = (uint16_t)min(lpD + P1, cap[p]);
                bp[D + 3] = (uint16_t)cap[p];
            }
        }
        __syncwarp();
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (!shift[p]) continue;
            const uint16_t* bp = buf + p * kBufLen;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q0 = min(max(s0 + 2 * j + sigma[p], -2), D + 1) + 2;
                const int q1 = min(max(s0 + 2 * j + 1 + sigma[p], -2), D + 1) + 2;
                T[p][j] = FM_IN(q0, D + 4, 0x301) && FM_IN(q1, D + 4, 0x301)
                              ? (uint32_t)bp[q0] | ((uint32_t)bp[q1] << 16) : 0u;
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const uint32_t M2 = dup2(Mp[p]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t v = first[p] ? Sv[j] : Sv[j] + T[p][j] - M2;
            L[p][j] = (v & q.vmask[j]) | (INF2 & ~q.vmask[j]);
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (q.variant == 2) {
            // key = cost << 8 | slot, one byte permutation per slot
            uint32_t key = 0xFFFFFFFFu;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                key = min(key, __byte_perm(L[p][j], (uint32_t)(q.s0 + 2 * j), 0x5104));
                key = min(key, __byte_perm(L[p][j], (uint32_t)(q.s0 + 2 * j + 1), 0x5324));
            }
            key = __reduce_min_sync(FULL, key);
            M[p] = key >> 8;
            wslot[p] = (int)(key & 255u);
        } else {
            const uint32_t mm = __vimin3_u16x2(__vimin3_u16x2(L[p][0], L[p][1], L[p][2]), L[p][3], L[p][3]);
            M[p] = __reduce_min_sync(FULL, min(mm & 0xFFFFu, mm >> 16));
            wslot[p] = 0;
        }
    }
}

// The path directions of a pass, as indices of the direction order of
// sgm.cu ((1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1)): horizontal,
// vertical, diagonal, anti-diagonal.  Pass B is pass A on the image turned by
// half a turn, so each of its directions is the opposite of pass A's.
__device__ __forceinline__ int dir_index(int pass, int which)
{
    return which == 0 ? pass : which == 1 ? 2 + pass : which == 2 ? 4 + pass : 7 - pass;
}

// the lane's part of a pixel's hypotheses: 8 slots at element offset `off`
__device__ __forceinline__ uint4 ld_slots(const uint16_t* base, size_t off)
{
    return __ldg(reinterpret_cast<const uint4*>(base + off));
}

// Winner-takes-all and sub-plane refinement (Sec. 2.3.4) of one pixel from its
// aggregate (the lane's slots in tot, two per register), as the stand-alone
// kernel does it: the lowest slot of least cost, the parabola through its
// neighbours' costs, the depth of the refined plane.
__device__ __forceinline__ void wave_wta(const WaveFrame& F, size_t pix, int x, int y, int lo_p,
                                         const uint32_t (&tot)[4], int D, int s0, int lane)
{
    uint32_t v[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = tot[j] & 0xFFFFu;
        v[2 * j + 1] = tot[j] >> 16;
    }
    uint32_t key = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (s0 + i < D) key = min(key, (v[i] << 8) | (uint32_t)(s0 + i));
    key = __reduce_min_sync(FULL, key);
    const int s = (int)(key & 255u);
    const int sm = max(s - 1, 0), sp = min(s + 1, D - 1);
    uint32_t vm = 0, vp = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((sm & 7) == i) vm = v[i];
        if ((sp & 7) == i) vp = v[i];
    }
    vm = __shfl_sync(FULL, vm, sm >> 3);
    vp = __shfl_sync(FULL, vp, sp >> 3);
    if (lane != 0) return;
    const int G = F.G;
    const int g = min(max(lo_p + s, 0), G - 1);
    const float x0 = __ldg(F.delta + g);
    float xs = x0;
    if (s > 0 && s < D - 1)
        xs = wta_vertex(x0, __ldg(F.delta + max(g - 1, 0)), __ldg(F.delta + min(g + 1, G - 1)), (float)(key >> 8),
                        (float)vm, (float)vp);
    if (FM_IN(pix, (size_t)F.a.W * F.a.H, 0x302)) F.depth[pix] = wta_depth(xs, x, y, F.K, F.n0, F.n1, F.n2);
    if (F.gwin) F.gwin[pix] = g;
}

// A predecessor in the row above: the lane's path costs (INF16 where the
// lane holds no slot), {minimum, winning plane, its predecessor's winning
// plane}, and the column's window start and image value.
struct Pred {
    uint4 L = make_uint4(INF2, INF2, INF2, INF2);
    int4 sc = make_int4(0, 0, 0, 0);
    int lo = 0, ip = 0;
};

// What a step needs of its pixel, loaded two columns ahead: the lane's data
// costs (and in pass B the lane's part of T1), the window start, the image
// value, and for the surface-normal variant the index jumps of the pass's
// four directions (one byte each).
struct PixIn {
    uint4 s, t;
    int lo, ip;
    uint32_t dsn;
};

template <int PASS>
__device__ __forceinline__ void load_pix(const WaveFrame& F, size_t pix, int x, int y, size_t soff, bool act,
                                         PixIn& o)
{
    const SgmArgs& a = F.a;
    if (act && FM_IN(pix * a.pstride + soff + 7, (size_t)a.W * a.H * a.pstride, 0x303)) {
        o.s = ld_slots(a.S, pix * a.pstride + soff);
        if (PASS) o.t = ld_slots(F.T1, pix * a.pstride + soff);
    }
    o.lo = a.lo ? __ldg(a.lo + pix) : 0;
    o.ip = a.use_lut ? (int)__ldg(a.img + (size_t)y * a.img_pitch + x) : 0;
    o.dsn = 0;
    if (a.variant == 1 && a.dI) {
        const size_t np = (size_t)a.W * a.H;
#pragma unroll
        for (int w = 0; w < 4; ++w)
            o.dsn |= (uint32_t)(uint8_t)__ldg(a.dI + (size_t)dir_index(PASS, w) * np + pix) << (8 * w);
    }
}

// One row of one pass, run by one warp.  Pass coordinates (xp, yp): pass A is
// the image, pass B the image turned by half a turn (x = W-1-xp, y = H-1-yp).
template <int PASS, bool EIGHT>
__device__ __forceinline__ void wave_row(const WaveFrame& F, int blk, int warp, int lane, WaveSmem& sm, int* err)
{
    const SgmArgs& a = F.a;
    const int W = a.W, H = a.H, D = a.D;
    const int yp = blk * R + warp;
    if (yp >= H) return;                   // warp-uniform; no row below waits on it
    if (!FM_IN(blk, F.nblocks, 0x305)) return;
    const int y = PASS ? H - 1 - yp : yp;
    // the row above is the previous warp of this CTA, or the last warp of the
    // CTA of the block above through the global ring; the row below likewise
    const bool up = yp > 0, up_global = up && warp == 0;
    const bool down = yp + 1 < H, down_global = down && warp == R - 1;
    int* flags = F.gflag + (PASS ? 2 * F.nblocks : 0);
    const int NR = F.ring;
    const uint4* gL_up = up_global ? F.gring + (size_t)(blk - 1) * NR * 3 * 32 : nullptr;
    const int4* gS_up = up_global ? F.gscal + (size_t)(blk - 1) * NR * 4 : nullptr;
    uint4* gL_dn = down_global ? F.gring + (size_t)blk * NR * 3 * 32 : nullptr;
    int4* gS_dn = down_global ? F.gscal + (size_t)blk * NR * 4 : nullptr;
    int* gf_up = up_global ? flags + 2 * (blk - 1) : nullptr;     // [0] published, [1] consumed
    int* gf_dn = down_global ? flags + 2 * blk : nullptr;

    PathIn q;
    q.D = D;
    q.s0 = lane * 8;
    q.lane = lane;
    q.variant = a.variant;
    q.p1 = a.p1;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        q.vmask[j] = ((q.s0 + 2 * j < D) ? 0xFFFFu : 0u) | ((q.s0 + 2 * j + 1 < D) ? 0xFFFF0000u : 0u);
    const bool act = q.s0 < D;
    const size_t soff = (size_t)(q.s0 >> a.bshift) * a.bstride + (q.s0 & ((1 << a.bshift) - 1));
    const size_t rowpix = (size_t)y * W;
    uint16_t* buf = sm.buf[warp];

    // the horizontal path's predecessor (the previous column of this row)
    uint32_t Lh[4] = {INF2, INF2, INF2, INF2};
    uint32_t Mh = 0;
    int g1h = 0, g2h = 0, lo_prev = 0, ip_prev = 0;
    // progress of the neighbouring rows as last seen
    int seen_up = 0, seen_dn = 0;

    auto xi = [&](int xp) { return PASS ? W - 1 - xp : xp; };
    PixIn c0, c1;
    c0.s = c0.t = c1.s = c1.t = make_uint4(0, 0, 0, 0);
    c1.lo = c1.ip = 0;
    c1.dsn = 0;
    load_pix<PASS>(F, rowpix + xi(0), xi(0), y, soff, act, c0);
    if (W > 1) load_pix<PASS>(F, rowpix + xi(1), xi(1), y, soff, act, c1);

    for (int xp = 0; xp < W; ++xp) {
        const int x = xi(xp);
        const size_t pix = rowpix + x;
        const PixIn cur = c0;
        c0 = c1;
        if (xp + 2 < W) load_pix<PASS>(F, rowpix + xi(xp + 2), xi(xp + 2), y, soff, act, c1);
        const int lo_p = cur.lo, ip = cur.ip;
        const uint32_t Sv[4] = {cur.s.x, cur.s.y, cur.s.z, cur.s.w};

        // ---- the row above: columns xp - 1 .. xp + 1 published
        Pred pv, pd, pa;
        if (up) {
            const int need = min(xp + 2, W);
            if (seen_up < need)
                seen_up = up_global ? wait_at_least<true>(gf_up, need, err, lane)
                                    : wait_at_least<false>(&sm.prog[warp - 1], need, err, lane);
            auto fetch = [&](int col, int w) {
                Pred o;
                int4 t;
                if (up_global) {
                    const int slot = col & (NR - 1);
                    if (act) o.L = __ldcg(gL_up + ((size_t)slot * 3 + w) * 32 + lane);
                    o.sc = __ldcg(gS_up + (size_t)slot * 4 + w);
                    t = __ldcg(gS_up + (size_t)slot * 4 + 3);
                } else {
                    const int slot = col & (NS - 1);
                    if (act) o.L = sm.L[warp - 1][slot][w][lane];
                    o.sc = sm.sc[warp - 1][slot][w];
                    t = sm.sc[warp - 1][slot][3];
                }
                o.lo = t.x;
                o.ip = t.y;
                return o;
            };
            pv = fetch(xp, 0);
            if (EIGHT) {
                if (xp > 0) pd = fetch(xp - 1, 1);
                if (xp + 1 < W) pa = fetch(xp + 1, 2);
            }
        }
        // ---- room in the ring towards the row below: the slot's previous
        // column (xp - NS, or xp - NR across CTAs) was last read by the row
        // below at its step xp - NS + 1 (never waits when NR > W)
        if (down) {
            const int need = xp - (down_global ? NR : NS) + 2;
            if (seen_dn < need)
                seen_dn = down_global ? wait_at_least<true>(gf_dn + 1, need, err, lane)
                                      : wait_at_least<false>(&sm.cons[warp + 1], need, err, lane);
        }

        // ---- the paths (Eq. xsgm), each added to the running total
        auto di_of = [&](int w, int g1, int g2, int step) {
            int di = 0;
            if (a.variant == 1) di = (int)(int8_t)(cur.dsn >> (8 * w));
            else if (a.variant == 2 && step >= 2) di = g2 - g1;
            return min(max(di, -a.dmax), a.dmax);
        };
        auto p2_of = [&](int ipred) {
            if (!a.use_lut) return a.p2;
            const int d = ip - ipred;
            return FM_IN(d < 0 ? -d : d, 256, 0x304) ? (int)a.lut[d < 0 ? -d : d] : 0;
        };
        uint32_t tot[4];
        if (PASS) {
            tot[0] = cur.t.x; tot[1] = cur.t.y; tot[2] = cur.t.z; tot[3] = cur.t.w;
        } else {
            tot[0] = tot[1] = tot[2] = tot[3] = 0u;
        }
        // the pass's paths in one batched step: p = 0 horizontal (the previous
        // column of this row), then the paths from the row above (vertical,
        // diagonal, anti-diagonal), whose steps from the path's start are yp,
        // min(xp, yp) and min(W-1-xp, yp)
        constexpr int NP = EIGHT ? 4 : 2;
        uint32_t Lp[NP][4], Mp[NP];
        bool first[NP];
        int sig[NP], p2v[NP], g1c[NP];
#pragma unroll
        for (int j = 0; j < 4; ++j) Lp[0][j] = Lh[j];
        Mp[0] = Mh;
        first[0] = xp == 0;
        sig[0] = first[0] ? 0 : lo_p - lo_prev + di_of(0, g1h, g2h, xp);
        p2v[0] = first[0] ? 0 : p2_of(ip_prev);
        g1c[0] = 0;
#pragma unroll
        for (int p = 1; p < NP; ++p) {
            const Pred& P = p == 1 ? pv : (p == 2 ? pd : pa);
            const bool have = p == 1 ? up : (p == 2 ? up && xp > 0 : up && xp + 1 < W);
            const int step = p == 1 ? yp : (p == 2 ? min(xp, yp) : min(W - 1 - xp, yp));
            first[p] = !have;
            const int g1 = have ? P.sc.y : 0, g2 = have ? P.sc.z : 0;
            g1c[p] = g1;
            Lp[p][0] = P.L.x; Lp[p][1] = P.L.y; Lp[p][2] = P.L.z; Lp[p][3] = P.L.w;
            Mp[p] = have ? (uint32_t)P.sc.x : 0u;
            sig[p] = have ? lo_p - P.lo + di_of(p, g1, g2, step) : 0;
            p2v[p] = have ? p2_of(P.ip) : 0;
        }
        uint32_t L[NP][4], M[NP];
        int ws[NP];
        paths_step<NP>(q, Sv, Lp, Mp, first, sig, p2v, buf, L, M, ws);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int j = 0; j < 4; ++j) tot[j] += L[p][j] & q.vmask[j];
#pragma unroll
        for (int j = 0; j < 4; ++j) Lh[j] = L[0][j];
        Mh = M[0];
        g2h = g1h;
        g1h = lo_p + ws[0];
        // the paths from the row above are published for the row below: the
        // lane's costs and {minimum, winning plane, the predecessor's winning
        // plane}
        const int pslot = xp & ((down_global ? NR : NS) - 1);
        if (down) {
#pragma unroll
            for (int p = 1; p < NP; ++p) {
                const int w = p - 1;
                const uint4 lv = make_uint4(L[p][0], L[p][1], L[p][2], L[p][3]);
                const int4 sc = make_int4((int)M[p], lo_p + ws[p], g1c[p], 0);
                if (down_global) {
                    if (act) __stcg(gL_dn + ((size_t)pslot * 3 + w) * 32 + lane, lv);
                    if (lane == 0) __stcg(gS_dn + (size_t)pslot * 4 + w, sc);
                } else {
                    if (act) sm.L[warp][pslot][w][lane] = lv;
                    if (lane == 0) sm.sc[warp][pslot][w] = sc;
                }
            }
        }
        lo_prev = lo_p;
        ip_prev = ip;
        // the column's window start and image value; then the flags: this
        // step is done with the row above's columns left of xp + 1, and the
        // column is published
        if (down && lane == 0) {
            const int4 cs = make_int4(lo_p, ip, 0, 0);
            if (down_global) __stcg(gS_dn + (size_t)pslot * 4 + 3, cs);
            else sm.sc[warp][pslot][3] = cs;
        }
        __syncwarp();
        const bool kg = ((xp + 1) & (KG - 1)) == 0 || xp + 1 == W;
        if (lane == 0) {
            if (up) {
                if (!up_global) st_release_cta(&sm.cons[warp], xp + 1);
                else if (kg) st_release_gpu(gf_up + 1, xp + 1);
            }
            if (down) {
                if (!down_global) st_release_cta(&sm.prog[warp], xp + 1);
                else if (kg) st_release_gpu(gf_dn, xp + 1);
            }
        }

        // ---- pass A: the sum of its paths; pass B: the aggregate and the winner
        const size_t off = pix * a.pstride + soff;
        // a lane that holds no hypothesis stores nothing (its offset is not checked)
        const bool oin = act && FM_IN(off + 7, (size_t)W * H * a.pstride, 0x306);
        if (!PASS) {
            if (act && oin) *reinterpret_cast<uint4*>(F.T1 + off) = make_uint4(tot[0], tot[1], tot[2], tot[3]);
        } else {
            if (a.Sbar && act && oin)
                *reinterpret_cast<uint4*>(a.Sbar + off) = make_uint4(tot[0], tot[1], tot[2], tot[3]);
            wave_wta(F, pix, x, y, lo_p, tot, D, q.s0, lane);
        }
    }
}

// Persistent CTAs: each takes the next block of rows (item) in launch order
// from the pass's ticket, so the block above an item is always running or
// done.  A block waits on the block below it only through a short ring; the
// launch is cooperative (every CTA resident), so with a frame's blocks no
// more than the CTAs the successor an item waits on is always taken; a frame
// with more blocks gets whole-row rings and never waits downwards.
template <int PASS, bool EIGHT>
__global__ void __launch_bounds__(R * 32, 4) sgm_wave_kernel(const __grid_constant__ WaveBatch b)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    WaveSmem& sm = *reinterpret_cast<WaveSmem*>(smraw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int total = b.item0[b.nframes];
    for (;;) {
        if (threadIdx.x == 0) sm.item = atomicAdd(b.ticket + PASS, 1);
        if (threadIdx.x < R) {
            sm.prog[threadIdx.x] = 0;
            sm.cons[threadIdx.x] = 0;
        }
        __syncthreads();
        const int item = sm.item;
        if (item >= total) break;
        int f = 0;
        while (f + 1 < b.nframes && b.item0[f + 1] <= item) ++f;
        wave_row<PASS, EIGHT>(b.f[f], item - b.item0[f], warp, lane, sm, b.err);
        __syncthreads();
    }
}

// the kernel of a pass and path count
using WaveKernel = void (*)(const WaveBatch);
WaveKernel wave_kernel(int pass, bool eight)
{
    return pass ? (eight ? sgm_wave_kernel<1, true> : sgm_wave_kernel<1, false>)
                : (eight ? sgm_wave_kernel<0, true> : sgm_wave_kernel<0, false>);
}

}  // namespace

FM_CHECK_TAKE(check_take_wave)

int wave_blocks(int H) { return (H + R - 1) / R; }
int wave_ring_cols(int W, int H, int cap)
{
    if (wave_blocks(H) <= cap) return NG;
    int r = NG;
    while (r < W + 1) r *= 2;
    return r;
}
size_t wave_ring_bytes(int W, int H, int cap, size_t* scal_off)
{
    const size_t cols = (size_t)wave_blocks(H) * wave_ring_cols(W, H, cap);
    const size_t L = cols * 3 * 32 * sizeof(uint4);
    if (scal_off) *scal_off = L;
    return L + cols * 4 * sizeof(int4);
}
size_t wave_flag_bytes(int H) { return (size_t)2 * 2 * wave_blocks(H) * sizeof(int); }

// CTAs of the two-pass kernels that fit on the device at once (0 when they
// cannot be launched cooperatively); the dynamic shared-memory limit is
// raised on first use
int wave_capacity(int device)
{
    static std::mutex mu;
    static std::map<int, int> cap;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cap.find(device);
    if (it != cap.end()) return it->second;
    int coop = 0, nsm = 0, occ = 1 << 30;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int smem = (int)sizeof(WaveSmem);
    bool ok = coop != 0;
    for (int i = 0; i < 4 && ok; ++i) {
        const WaveKernel k = wave_kernel(i & 1, i >> 1);
        int o = 0;
        ok = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, R * 32, smem) == cudaSuccess;
        occ = std::min(occ, o);
    }
    cudaGetLastError();
    const int c = ok ? nsm * occ : 0;
    cap[device] = c;
    return c;
}

void launch_sgm_wave(const WaveBatch& b, int pass, int ctas, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(R * 32);
    cfg.dynamicSmemBytes = sizeof(WaveSmem);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // the frames of a batch share the configuration, so its path count
    cudaLaunchKernelEx(&cfg, wave_kernel(pass, b.f[0].a.paths == 8), b);
    count_launch();
}

}  // namespace fm
