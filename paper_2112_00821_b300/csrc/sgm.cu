// Surface-aware semi-global matching (Sec. 2.3 of FaSS-MVS) for sm_103a.
//
// One warp walks one path line; lane l holds hypotheses 8l .. 8l+7 of the
// current pixel, so the previous path line stays in registers.  Per step:
// the transition minimum T(s') = min(L'(s'), L'(s' +- 1) + P1, M' + P2) is
// formed on the predecessor's slots (two neighbour shuffles), shifted by the
// warp-uniform sigma = lo_p - lo_{p-r} + di through a per-warp shared buffer
// when sigma != 0, added to the data cost, and the new minimum (and, for the
// path-gradient variant, its slot) comes from a 5-step shuffle reduction.
// Each direction is one launch; the first writes the aggregate, the others
// add to it (stream order keeps them apart).
#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int WARPS = 4;
constexpr uint32_t INF = 0x3FFFFFFFu;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ void unpack8(uint4 v, uint32_t (&o)[8])
{
    o[0] = v.x & 0xFFFFu; o[1] = v.x >> 16;
    o[2] = v.y & 0xFFFFu; o[3] = v.y >> 16;
    o[4] = v.z & 0xFFFFu; o[5] = v.z >> 16;
    o[6] = v.w & 0xFFFFu; o[7] = v.w >> 16;
}

__device__ __forceinline__ uint4 pack8(const uint32_t (&o)[8])
{
    return make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16),
                      o[6] | (o[7] << 16));
}

__global__ void __launch_bounds__(WARPS * 32)
sgm_dir_kernel(const SgmArgs a, int r, int dx, int dy, int nlines, int first)
{
    __shared__ uint32_t sT[WARPS][kMaxSlots + 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int line = blockIdx.x * WARPS + warp;
    if (line >= nlines) return;                // warp-uniform
    const int W = a.W, H = a.H, D = a.D;
    int x, y;
    if (dy == 0) { x = dx > 0 ? 0 : W - 1; y = line; }
    else if (dx == 0) { y = dy > 0 ? 0 : H - 1; x = line; }
    else if (line < H) { x = dx > 0 ? 0 : W - 1; y = line; }
    else { int i = line - H; y = dy > 0 ? 0 : H - 1; x = dx > 0 ? i + 1 : W - 2 - i; }

    const int s0 = lane * 8;
    const bool act = s0 < D;
    uint32_t Lp[8], L[8], Sv[8];
    uint32_t M = 0;
    int g1 = 0, g2 = 0;       // winning plane of p - r and p - 2r (path gradient)
    int lo_prev = 0;
    int ipix_prev = 0;
    const size_t plane_stride = (size_t)W * H;

    uint4 sraw = make_uint4(0, 0, 0, 0);
    if (act) sraw = __ldg(reinterpret_cast<const uint4*>(a.S + ((size_t)y * W + x) * a.Ds + s0));

    for (int step = 0; x >= 0 && x < W && y >= 0 && y < H; ++step, x += dx, y += dy) {
        const size_t pix = (size_t)y * W + x;
        unpack8(sraw, Sv);
        // prefetch the next pixel's costs
        const int nx = x + dx, ny = y + dy;
        if (act && nx >= 0 && nx < W && ny >= 0 && ny < H)
            sraw = __ldg(reinterpret_cast<const uint4*>(a.S + ((size_t)ny * W + nx) * a.Ds + s0));
        uint4 acc_raw = make_uint4(0, 0, 0, 0);
        if (!first && act) acc_raw = *reinterpret_cast<const uint4*>(a.Sbar + pix * a.Ds + s0);

        const int lo_p = a.lo ? __ldg(a.lo + pix) : 0;
        if (step == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) L[i] = (s0 + i < D) ? Sv[i] : INF;
        } else {
            int di = 0;
            if (a.variant == 1 && a.dI) di = a.dI[(size_t)r * plane_stride + pix];
            else if (a.variant == 2 && step >= 2) di = g2 - g1;
            di = min(max(di, -a.dmax), a.dmax);
            const int sigma = lo_p - lo_prev + di;
            int P2 = a.p2;
            if (a.use_lut) {
                int d = (int)__ldg(a.img + (size_t)y * a.img_pitch + x) - ipix_prev;
                P2 = a.lut[d < 0 ? -d : d];
            }
            P2 = max(P2, a.p1);
            const uint32_t P1 = (uint32_t)a.p1;
            const uint32_t cap = M + (uint32_t)P2;
            uint32_t left = __shfl_up_sync(FULL, Lp[7], 1);
            uint32_t right = __shfl_down_sync(FULL, Lp[0], 1);
            if (lane == 0) left = INF;
            if (lane == 31) right = INF;
            uint32_t T[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                uint32_t pv = i == 0 ? left : Lp[i - 1];
                uint32_t nv = i == 7 ? right : Lp[i + 1];
                T[i] = min(min(Lp[i], cap), min(pv, nv) + P1);
            }
            if (sigma != 0) {
                uint32_t* buf = sT[warp];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (s0 + i < D) buf[1 + s0 + i] = T[i];
                if (lane == 0) buf[0] = min(Lp[0] + P1, cap);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (s0 + i == D - 1) buf[D + 1] = min(Lp[i] + P1, cap);
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    int q = s0 + i + sigma;
                    T[i] = (q >= -1 && q <= D) ? buf[q + 1] : cap;
                }
                __syncwarp();
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) L[i] = (s0 + i < D) ? Sv[i] + T[i] - M : INF;
        }
        // new minimum (and its slot, lowest on ties)
        uint32_t key = 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (s0 + i < D) key = min(key, (L[i] << 8) | (uint32_t)(s0 + i));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(FULL, key, o));
        M = key >> 8;
        g2 = g1;
        g1 = lo_p + (int)(key & 255u);
        // accumulate
        if (act) {
            uint32_t o[8];
            if (first) {
#pragma unroll
                for (int i = 0; i < 8; ++i) o[i] = (s0 + i < D) ? (L[i] & 0xFFFFu) : 0u;
            } else {
                unpack8(acc_raw, o);
#pragma unroll
                for (int i = 0; i < 8; ++i) o[i] = (s0 + i < D) ? ((o[i] + L[i]) & 0xFFFFu) : o[i];
            }
            *reinterpret_cast<uint4*>(a.Sbar + pix * a.Ds + s0) = pack8(o);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) Lp[i] = L[i];
        lo_prev = lo_p;
        if (a.use_lut) ipix_prev = __ldg(a.img + (size_t)y * a.img_pitch + x);
    }
}

const int kDX[8] = {1, -1, 0, 0, 1, -1, 1, -1};
const int kDY[8] = {0, 0, 1, -1, 1, -1, -1, 1};

}  // namespace

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
