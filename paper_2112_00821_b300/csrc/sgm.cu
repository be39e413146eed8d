// Surface-aware semi-global matching (Sec. 2.3 of FaSS-MVS) for sm_103a.
//
// One warp walks one path line; lane l holds hypotheses 8l .. 8l+7 of the
// current pixel, two per register, so the previous step stays in registers.
// Per step: the transition minimum T(s') = min(L'(s'), L'(s' +- 1) + P1,
// M' + P2) is formed on the predecessor's slots with the packed 16x2 min and
// add-min instructions (the neighbour pairs across lanes come from two
// shuffles of the previous step), shifted by the warp-uniform
// sigma = lo_p - lo_{p-r} + di through a per-warp shared buffer when
// sigma != 0, and added to the data cost; the new minimum (and, for the
// path-gradient variant, its slot) comes from one warp min-reduction.
// The stage entry point runs one launch per direction, the first writing the
// aggregate and the others adding to it (stream order keeps them apart); the
// estimate runs several directions of several frames in one launch, each
// direction into its own partial sum, which the winner-takes-all step adds.
#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int WARPS = 4;
constexpr unsigned FULL = 0xFFFFFFFFu;

// The data costs and running aggregate of the pixel PF steps down the line
// are copied into a per-warp shared ring with cp.async (each lane its own 16
// bytes, so a per-thread wait suffices); the small per-pixel values (window
// start, image value, surface-normal jump) are prefetched in registers, a
// block of PF steps at a time.  A short ring and at most 80 registers (71
// used) let six or more CTAs (24 warps, i.e. 24 path lines) share an SM: more
// lines in flight hide the step-to-step latency better than a deeper
// prefetch (measured: PF 4 / 6 CTAs 15 % faster than PF 8 / 4 CTAs on the
// 1080p estimate).
constexpr int PF = 4;

struct StepScal {
    int lo, ipix, dsn;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void load_scal(const SgmArgs& a, int r, int x, int y, StepScal& o)
{
    const size_t pix = (size_t)y * a.W + x;
    if (!FM_IN(x, a.W, 0x205) || !FM_IN(y, a.H, 0x205)) { o.lo = o.ipix = o.dsn = 0; return; }
    o.lo = a.lo ? __ldg(a.lo + pix) : 0;
    o.ipix = a.use_lut ? (int)__ldg(a.img + (size_t)y * a.img_pitch + x) : 0;
    o.dsn = (a.variant == 1 && a.dI) ? (int)a.dI[(size_t)r * a.W * a.H + pix] : 0;
}

// Two hypotheses per 32-bit register: every path cost stays below 2^13 (the
// host checks paths * (max S + max P2) < 2^16), so packed values never carry
// or borrow across the halves; INF16 marks slots outside the window.
constexpr uint32_t INF16 = 0x3FFFu;
constexpr uint32_t INF2 = INF16 | (INF16 << 16);

__device__ __forceinline__ uint32_t dup2(uint32_t v) { return v | (v << 16); }

// One path line of direction r (line index in the order described at the
// launcher), run by one warp with its private shared buffers.
__device__ __forceinline__ void sgm_line(const SgmArgs& a, uint16_t* __restrict__ Sb, int r, int dx, int dy,
                                         int line, int first, uint16_t* buf, uint4 (*rg)[2][32])
{
    const int lane = threadIdx.x & 31;
    const int W = a.W, H = a.H, D = a.D;
    int x0, y0;
    if (dy == 0) { x0 = dx > 0 ? 0 : W - 1; y0 = line; }
    else if (dx == 0) { y0 = dy > 0 ? 0 : H - 1; x0 = line; }
    else if (line < H) { x0 = dx > 0 ? 0 : W - 1; y0 = line; }
    else { int i = line - H; y0 = dy > 0 ? 0 : H - 1; x0 = dx > 0 ? i + 1 : W - 2 - i; }
    int n = 1 << 30;                           // steps until the path leaves the image
    if (dx > 0) n = min(n, W - x0);
    if (dx < 0) n = min(n, x0 + 1);
    if (dy > 0) n = min(n, H - y0);
    if (dy < 0) n = min(n, y0 + 1);

    const int s0 = lane * 8;
    const bool act = s0 < D;
    // offset of this lane's slots s0 .. s0 + 7 within a pixel's hypotheses
    const size_t soff = (size_t)(s0 >> a.bshift) * a.bstride + (s0 & ((1 << a.bshift) - 1));
    // valid-slot masks per packed pair
    uint32_t vmask[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        vmask[j] = ((s0 + 2 * j < D) ? 0xFFFFu : 0u) | ((s0 + 2 * j + 1 < D) ? 0xFFFF0000u : 0u);
    uint32_t Lp[4];
    uint32_t left = INF2, right = INF2;        // neighbour pairs of the previous step
    uint32_t M = 0;
    int g1 = 0, g2 = 0;                        // winning plane of p - r and p - 2r (path gradient)
    int lo_prev = 0, ipix_prev = 0;
    const uint32_t P1 = (uint32_t)a.p1, P1P1 = dup2(P1);

    // per-step scalars (window start, intensity, index jump) are fetched PF
    // steps ahead and spread over the lanes: lane u holds those of the steps
    // congruent to u modulo PF, broadcast when the step comes
    // (double-buffered: at the start of each block of PF steps lanes 0 .. PF-1
    // fetch the next block's, so that one lane-divergent load serves PF steps)
    StepScal q{0, 0, 0}, qn{0, 0, 0};
    if (lane < PF && lane < n) load_scal(a, r, x0 + lane * dx, y0 + lane * dy, qn);
#pragma unroll
    for (int u = 0; u < PF; ++u) {
        if (u < n) {
            const int xx = x0 + u * dx, yy = y0 + u * dy;
            const size_t pp = ((size_t)yy * W + xx) * a.pstride + soff;
            if (act && FM_IN(pp + 7, (size_t)W * H * a.pstride, 0x201)) {
                cp_async16(&rg[u][0][lane], a.S + pp);
                if (!first) cp_async16(&rg[u][1][lane], Sb + pp);
            }
        }
        cp_async_commit();
    }

    // element offsets of the step's pixel and of the step PF ahead; a step moves
    // them by dstep
    const ptrdiff_t dstep = ((ptrdiff_t)dy * W + dx) * (ptrdiff_t)a.pstride;
    ptrdiff_t off = (ptrdiff_t)(((size_t)y0 * W + x0) * a.pstride + soff);
    ptrdiff_t pf_off = off + PF * dstep;
    for (int base = 0; base < n; base += PF) {
        q = qn;
        if (lane < PF && base + PF + lane < n)
            load_scal(a, r, x0 + (base + PF + lane) * dx, y0 + (base + PF + lane) * dy, qn);
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            const int step = base + u;
            if (step >= n) break;              // warp-uniform
            const int lo_p = __shfl_sync(FULL, q.lo, u);
            const int pk = __shfl_sync(FULL, (q.ipix & 0xFF) | (q.dsn * 256), u);
            const int cur_ipix = pk & 0xFF, cur_dsn = pk >> 8;
            cp_async_wait<PF - 1>();           // this step's group has landed
            const uint4 sraw = rg[u][0][lane];
            const uint4 acc = rg[u][1][lane];
            __syncwarp();
            if (step + PF < n && act && FM_IN(pf_off + 7, (size_t)W * H * a.pstride, 0x201)) {
                cp_async16(&rg[u][0][lane], a.S + pf_off);
                if (!first) cp_async16(&rg[u][1][lane], Sb + pf_off);
            }
            cp_async_commit();
            const uint32_t Sv[4] = {sraw.x, sraw.y, sraw.z, sraw.w};
            uint32_t L[4];
            if (step == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) L[j] = (Sv[j] & vmask[j]) | (INF2 & ~vmask[j]);
            } else {
                int di = 0;
                if (a.variant == 1) di = cur_dsn;
                else if (a.variant == 2 && step >= 2) di = g2 - g1;
                di = min(max(di, -a.dmax), a.dmax);
                const int sigma = lo_p - lo_prev + di;
                int P2 = a.p2;
                if (a.use_lut) {
                    int d = cur_ipix - ipix_prev;
                    P2 = FM_IN(d < 0 ? -d : d, 256, 0x204) ? a.lut[d < 0 ? -d : d] : 0;
                }
                P2 = max(P2, a.p1);
                const uint32_t cap = M + (uint32_t)P2, cap2 = dup2(cap);
                // T(s') = min(L'(s'), L'(s'-1) + P1, L'(s'+1) + P1, M + P2), packed,
                // with the 16x2 dynamic-programming min / add-min instructions
                uint32_t T[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t pv = __byte_perm(j == 0 ? left : Lp[j - 1], Lp[j], 0x5432);
                    const uint32_t nv = __byte_perm(Lp[j], j == 3 ? right : Lp[j + 1], 0x5432);
                    T[j] = __vimin3_u16x2(Lp[j], cap2, __viaddmin_u16x2(pv, P1P1, nv + P1P1));
                }
                if (sigma != 0) {
                    // shift by sigma slots through shared memory: index k + 2 holds
                    // T(k) for k in [-2, D+1]; beyond the predecessor's window the
                    // transition costs M + P2 (k = -2, D + 1 and clamped indices)
                    uint32_t* b32 = reinterpret_cast<uint32_t*>(buf);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (s0 + 2 * j + 1 < D) b32[1 + (s0 >> 1) + j] = T[j];
                        else if (s0 + 2 * j < D) buf[2 + s0 + 2 * j] = (uint16_t)(T[j] & 0xFFFFu);
                    }
                    const uint32_t lp0 = __shfl_sync(FULL, Lp[0], 0) & 0xFFFFu;
                    const int lastl = (D - 1) >> 3, lasti = (D - 1) & 7;
                    // Lp[lasti >> 1] by selects (an indexed read would go to local memory)
                    const uint32_t l01 = (lasti & 2) ? Lp[1] : Lp[0], l23 = (lasti & 2) ? Lp[3] : Lp[2];
                    const uint32_t lsel = (lasti & 4) ? l23 : l01;
                    const uint32_t lpw = __shfl_sync(FULL, lsel, lastl);
                    const uint32_t lpD = (lasti & 1) ? (lpw >> 16) : (lpw & 0xFFFFu);
                    if (lane == 0) {
                        buf[0] = (uint16_t)cap;
                        buf[1] = (uint16_t)min(lp0 + P1, cap);
                        buf[D + 2] = (uint16_t)min(lpD + P1, cap);
                        buf[D + 3] = (uint16_t)cap;
                    }
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int q0 = min(max(s0 + 2 * j + sigma, -2), D + 1) + 2;
                        const int q1 = min(max(s0 + 2 * j + 1 + sigma, -2), D + 1) + 2;
                        T[j] = FM_IN(q0, D + 4, 0x202) && FM_IN(q1, D + 4, 0x202)
                                   ? (uint32_t)buf[q0] | ((uint32_t)buf[q1] << 16) : 0u;
                    }
                    __syncwarp();
                }
                const uint32_t M2 = dup2(M);
#pragma unroll
                for (int j = 0; j < 4; ++j) L[j] = ((Sv[j] + T[j] - M2) & vmask[j]) | (INF2 & ~vmask[j]);
            }
            // neighbours for the next step, then the new minimum over the window
            // (with its lowest slot for the path gradient) by a warp reduction
            left = __shfl_up_sync(FULL, L[3], 1);
            right = __shfl_down_sync(FULL, L[0], 1);
            if (lane == 0) left = INF2;
            if (lane == 31) right = INF2;
            if (a.variant == 2) {
                // key = cost << 8 | slot: one byte permutation per slot takes
                // the slot number (byte 0) and the 16-bit cost (bytes 1, 2) with
                // a zero top byte
                uint32_t key = 0xFFFFFFFFu;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    key = min(key, __byte_perm(L[j], (uint32_t)(s0 + 2 * j), 0x5104));
                    key = min(key, __byte_perm(L[j], (uint32_t)(s0 + 2 * j + 1), 0x5324));
                }
                key = __reduce_min_sync(FULL, key);
                M = key >> 8;
                g2 = g1;
                g1 = lo_p + (int)(key & 255u);
            } else {
                const uint32_t mm = __vimin3_u16x2(__vimin3_u16x2(L[0], L[1], L[2]), L[3], L[3]);
                M = __reduce_min_sync(FULL, min(mm & 0xFFFFu, mm >> 16));
            }
            if (act) {
                uint4 o;
                if (first) {
                    o = make_uint4(L[0] & vmask[0], L[1] & vmask[1], L[2] & vmask[2], L[3] & vmask[3]);
                } else {
                    o = make_uint4(acc.x + (L[0] & vmask[0]), acc.y + (L[1] & vmask[1]),
                                   acc.z + (L[2] & vmask[2]), acc.w + (L[3] & vmask[3]));
                }
                if (FM_IN(off + 7, (size_t)W * H * a.pstride, 0x203)) *reinterpret_cast<uint4*>(Sb + off) = o;
            }
            off += dstep;
            pf_off += dstep;
#pragma unroll
            for (int j = 0; j < 4; ++j) Lp[j] = L[j];
            lo_prev = lo_p;
            ipix_prev = cur_ipix;
        }
    }
}

__global__ void __launch_bounds__(WARPS * 32, 6)
sgm_dir_kernel(const SgmArgs a, int r, int dx, int dy, int nlines, int first)
{
    __shared__ uint16_t sT[WARPS][kMaxSlots + 4];
    __shared__ uint4 ring[WARPS][PF][2][32];   // [step][S, S_bar][lane]
    const int warp = threadIdx.x >> 5;
    const int line = blockIdx.x * WARPS + warp;
    if (line >= nlines) return;                // warp-uniform
    sgm_line(a, a.Sbar, r, dx, dy, line, first, sT[warp], ring[warp]);
}

// Several directions of several frames in one launch.  Direction slot j of
// the launch runs direction b.r[j] into partial sum b.part[j] of every frame
// (b.first[j]: the slot writes that part instead of adding to it); the lines
// of (slot j, frame f) start at CTA line b.seg[j][f], each range padded to
// whole CTAs so the slot and frame are uniform across a CTA.  The arguments
// are one by-value kernel parameter (grid constant, so indexed reads stay in
// the constant bank).
__global__ void __launch_bounds__(WARPS * 32, 6)
sgm_batch_dir_kernel(const __grid_constant__ SgmBatch b)
{
    __shared__ uint16_t sT[WARPS][kMaxSlots + 4];
    __shared__ uint4 ring[WARPS][PF][2][32];
    const int cta_line = blockIdx.x * WARPS;
    int j = 0;
    while (j + 1 < b.nslots && b.seg[j + 1][0] <= cta_line) ++j;
    int f = 0;
    while (f + 1 < b.nframes && b.seg[j][f + 1] <= cta_line) ++f;
    const SgmArgs& a = b.a[f];
    const int r = b.r[j], dx = b.dx[j], dy = b.dy[j];
    const int warp = threadIdx.x >> 5;
    const int line = cta_line - b.seg[j][f] + warp;
    const int nlines = dy == 0 ? a.H : (dx == 0 ? a.W : a.W + a.H - 1);
    if (line >= nlines) return;                 // warp-uniform
    sgm_line(a, a.Sbar + (size_t)b.part[j] * a.part_stride, r, dx, dy, line, b.first[j], sT[warp], ring[warp]);
}

const int kDX[8] = {1, -1, 0, 0, 1, -1, 1, -1};
const int kDY[8] = {0, 0, 1, -1, 1, -1, -1, 1};

}  // namespace

int sgm_lines(int W, int H, int r)
{
    const int dx = kDX[r], dy = kDY[r];
    const int n = dy == 0 ? H : (dx == 0 ? W : W + H - 1);
    return (n + WARPS - 1) / WARPS * WARPS;     // whole CTAs per frame
}

FM_CHECK_TAKE(check_take_sgm)

void sgm_dir_of(int r, int* dx, int* dy)
{
    *dx = kDX[r];
    *dy = kDY[r];
}

void launch_sgm_batch(const SgmBatch& b, cudaStream_t st)
{
    const int blocks = b.seg[b.nslots - 1][b.nframes] / WARPS;
    if (blocks == 0) return;
    sgm_batch_dir_kernel<<<blocks, WARPS * 32, 0, st>>>(b);
    count_launch();
}

void launch_sgm(const SgmArgs& a, cudaStream_t st)
{
    for (int r = 0; r < a.paths; ++r) {
        int dx = kDX[r], dy = kDY[r];
        int nlines = dy == 0 ? a.H : (dx == 0 ? a.W : a.W + a.H - 1);
        int blocks = (nlines + WARPS - 1) / WARPS;
        sgm_dir_kernel<<<blocks, WARPS * 32, 0, st>>>(a, r, dx, dy, nlines, r == 0);
        count_launch();
    }
}

}  // namespace fm
