// Plane-sweep census cost volume (Alg. 1 of FaSS-MVS) for sm_103a.
//
// One CTA owns a 32 x 8 tile of reference pixels and walks the planes its
// windows need, eight planes per batch (one warp per plane).  For each view
// the eight warped 40 x 14 sample tiles (tile + census halo) are produced
// into shared memory, then every warp builds the 9x7 census strings of its
// plane for the 8 pixels of its lane's column, XORs them with the reference
// census and accumulates the left / right subset sums in registers.
//
// Sampling reading (shared with the oracle, stated in the header): the
// homography is evaluated in double-float arithmetic (two FP32 words) so the
// 1/256-pixel fixed-point position floor(256 u) agrees with an FP64
// evaluation except within ~1e-10 px of a grid line; the bilinear blend is
// exact integer arithmetic with 8-bit weights.
#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int TX = 32, TY = 8;          // pixel tile
constexpr int SX = TX + 8, SY = TY + 6; // sample tile with the 9x7 halo
constexpr int PB = 8;                   // planes per batch (= warps)
constexpr int THREADS = 256;
constexpr int RUN = SX / 2;             // samples per sampling task (one half row)
constexpr int PMAX = 1 << 24;

struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    float h = __fadd_rn(s.hi, lo);
    return {h, __fsub_rn(lo, __fsub_rn(h, s.hi))};
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

// floor(256 * N / Dn) clamped to [-2^24, 2^24], for Dn > 0.  q = N/D to a few
// ulps, then the residual N - q D in double-float gives the correction.
__device__ __forceinline__ int fix_pos(df N, df Dn)
{
    float r = rcp_approx(Dn.hi);
    float q = __fmul_rn(N.hi, r);
    float e1 = __fmaf_rn(-q, Dn.hi, N.hi);
    float e2 = __fmaf_rn(-q, Dn.lo, N.lo);
    float corr = __fmul_rn(__fadd_rn(e1, e2), r);
    float a = __fmul_rn(q, 256.0f);
    a = fminf(fmaxf(a, -17000000.0f), 17000000.0f);
    float af = floorf(a);
    float rem = __fadd_rn(__fsub_rn(a, af), __fmul_rn(corr, 256.0f));
    int P = (int)af + (int)floorf(rem);
    return min(max(P, -PMAX), PMAX);
}

__device__ __forceinline__ df load_df(const float* h, int i) { return {h[i], h[9 + i]}; }

// warped sample value of image img (W x H, pitch) at the fixed-point position
__device__ __forceinline__ int bilinear_fix(const uint8_t* __restrict__ img, int W, int H, int pitch,
                                            int Pu, int Pv)
{
    int cu = min(max(Pu, 0), 256 * (W - 1));
    int cv = min(max(Pv, 0), 256 * (H - 1));
    int iu = min(cu >> 8, W - 2);
    int iv = min(cv >> 8, H - 2);
    int A = cu - 256 * iu, B = cv - 256 * iv;
    const uint8_t* r0 = img + (size_t)iv * pitch + iu;
    int i00 = __ldg(r0), i01 = __ldg(r0 + 1);
    int i10 = __ldg(r0 + pitch), i11 = __ldg(r0 + pitch + 1);
    int top = i00 * (256 - A) + i01 * A;
    int bot = i10 * (256 - A) + i11 * A;
    return top * (256 - B) + bot * B;
}

__global__ void __launch_bounds__(THREADS, 2)
cost_kernel(const CostArgs a)
{
    __shared__ int32_t sV[PB][SY][SX];
    __shared__ uint8_t sOk[PB][TY][TX];
    __shared__ int s_glo, s_ghi;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * TY;
    const int W = a.W, H = a.H;

    // plane range needed by this tile: union of [lo_p, lo_p + D)
    if (tid == 0) { s_glo = a.G; s_ghi = 0; }
    __syncthreads();
    {
        int px = tx0 + (tid & 31), py = ty0 + (tid >> 5);
        if (px < W && py < H) {
            int l = a.lo ? a.lo[(size_t)py * W + px] : 0;
            atomicMin(&s_glo, l);
            atomicMax(&s_ghi, l + a.D);
        }
    }
    __syncthreads();
    const int glo = max(s_glo, 0), ghi = min(s_ghi, a.G);   // guards against an out-of-range window map

    // this lane's column of 8 pixels: reference census and windows
    const int px = tx0 + lane;
    uint32_t rlo[TY], rhi[TY];
    int plo[TY];
#pragma unroll
    for (int r = 0; r < TY; ++r) {
        int py = ty0 + r;
        bool in = px < W && py < H;
        uint64_t c = in ? a.cref[(size_t)py * W + px] : 0ull;
        rlo[r] = (uint32_t)c;
        rhi[r] = (uint32_t)(c >> 32);
        plo[r] = in ? (a.lo ? a.lo[(size_t)py * W + px] : 0) : (1 << 30);
    }

    for (int g0 = glo; g0 < ghi; g0 += PB) {
        uint32_t acc[TY];   // left sum in the low half, right sum in the high half
#pragma unroll
        for (int r = 0; r < TY; ++r) acc[r] = 0;

        for (int k = 0; k < a.V; ++k) {
            // ---- sampling: 8 planes x 14 rows x 2 half rows = 224 tasks
            if (tid < PB * SY * 2) {
                const int b = tid / (SY * 2);
                const int row = (tid % (SY * 2)) >> 1;
                const int half = tid & 1;
                const int g = g0 + b;
                if (g < ghi) {
                    const float* h = a.htab + ((size_t)g * a.V + k) * 18;
                    const int y = min(max(ty0 - 3 + row, 0), H - 1);
                    const int xs = tx0 - 4 + half * RUN;
                    int xc = min(max(xs, 0), W - 1);
                    const float fx = (float)xc, fy = (float)y;
                    df Nu = df_add(df_add(df_mul_int(load_df(h, 0), fx), df_mul_int(load_df(h, 1), fy)), load_df(h, 2));
                    df Nv = df_add(df_add(df_mul_int(load_df(h, 3), fx), df_mul_int(load_df(h, 4), fy)), load_df(h, 5));
                    df Dn = df_add(df_add(df_mul_int(load_df(h, 6), fx), df_mul_int(load_df(h, 7), fy)), load_df(h, 8));
                    const df h0 = load_df(h, 0), h3 = load_df(h, 3), h6 = load_df(h, 6);
                    const uint8_t* img = a.views.img[k];
#pragma unroll 4
                    for (int j = 0; j < RUN; ++j) {
                        int x = xs + j;
                        if (j > 0 && x >= 1 && x <= W - 1) {
                            Nu = df_add(Nu, h0);
                            Nv = df_add(Nv, h3);
                            Dn = df_add(Dn, h6);
                        }
                        bool front = Dn.hi > 0.0f || (Dn.hi == 0.0f && Dn.lo > 0.0f);
                        int Pu = -PMAX, Pv = -PMAX;
                        if (front) {
                            Pu = fix_pos(Nu, Dn);
                            Pv = fix_pos(Nv, Dn);
                        }
                        const int sx = half * RUN + j;
                        sV[b][row][sx] = bilinear_fix(img, W, H, a.pitch, Pu, Pv);
                        if (row >= 3 && row < 3 + TY && sx >= 4 && sx < 4 + TX) {
                            bool ok = front && Pu >= 0 && Pu <= 256 * (W - 1) && Pv >= 0 &&
                                      Pv <= 256 * (H - 1);
                            sOk[b][row - 3][sx - 4] = ok;
                        }
                    }
                }
            }
            __syncthreads();

            // ---- census + Hamming: warp = plane, lane = column, 8 pixels
            const int g = g0 + warp;
            if (g < ghi) {
                uint32_t cen[TY], blo[TY], bhi[TY];
#pragma unroll
                for (int r = 0; r < TY; ++r) {
                    cen[r] = (uint32_t)sV[warp][r + 3][lane + 4];
                    blo[r] = 0;
                    bhi[r] = 0;
                }
#pragma unroll
                for (int j = 0; j < SY; ++j) {
                    uint32_t v[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) v[i] = (uint32_t)sV[warp][j][lane + i];
#pragma unroll
                    for (int r = 0; r < TY; ++r) {
                        const int dy = j - r;
                        if (dy < 0 || dy > 6) continue;
#pragma unroll
                        for (int i = 0; i < 9; ++i) {
                            const int kb = dy * 9 + i;
                            uint32_t bit = v[i] < cen[r] ? 1u : 0u;
                            if (kb < 32) blo[r] |= bit << kb;
                            else bhi[r] |= bit << (kb - 32);
                        }
                    }
                }
                const int sh = a.views.side[k] < 0 ? 0 : 16;
#pragma unroll
                for (int r = 0; r < TY; ++r) {
                    uint32_t hcost = __popc(blo[r] ^ rlo[r]) + __popc(bhi[r] ^ rhi[r]);
                    if (!sOk[warp][r][lane]) hcost = kCensusMax;
                    acc[r] += hcost << sh;
                }
            }
            __syncthreads();
        }

        // ---- left/right combination and store
        const int g = g0 + warp;
        if (g < ghi && px < W) {
#pragma unroll
            for (int r = 0; r < TY; ++r) {
                const int py = ty0 + r;
                const int s = g - plo[r];
                if (py < H && s >= 0 && s < a.D) {
                    uint32_t sl = acc[r] & 0xFFFFu, sr = acc[r] >> 16;
                    uint32_t vl = 0xFFFFFFFFu, vr = 0xFFFFFFFFu;
                    // round-half-up rescaling to nmax images: (s*nmax + n/2) / n
                    // (x * ceil(2^32 / n)) >> 32 == x / n exactly for x < 2^16, n <= 16
                    if (a.nL > 0) vl = (uint32_t)(((uint64_t)(sl * a.nmax + (a.nL >> 1)) * a.mL) >> 32);
                    if (a.nR > 0) vr = (uint32_t)(((uint64_t)(sr * a.nmax + (a.nR >> 1)) * a.mR) >> 32);
                    a.S[((size_t)py * W + px) * a.Ds + s] = (uint16_t)min(vl, vr);
                }
            }
        }
    }
}

}  // namespace

void launch_cost(const CostArgs& a, cudaStream_t st)
{
    dim3 grid((a.W + TX - 1) / TX, (a.H + TY - 1) / TY);
    cost_kernel<<<grid, THREADS, 0, st>>>(a);
    count_launch();
}

// ---------------------------------------------------------------- level tables
namespace {
__global__ void prep_level_kernel(const ViewGeom vg, const LevelPlanes lp, float* htab,
                                  float* delta)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= lp.G * lp.V) return;
    int g = i / lp.V, k = i % lp.V;
    double rho = lp.rho0 + (double)g * lp.drho;
    float* o = htab + (size_t)i * 18;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double h = vg.A[k][3 * r + c] - rho * vg.e[k][r] * vg.c[k][c];
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
