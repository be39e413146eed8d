// Per-pixel stages of the FaSS-MVS hot path for sm_103a: Gaussian pyramid
// (Sec. 2.1), reference census (Sec. 2.2.1), winner-takes-all with sub-plane
// refinement (Eq. sgm-wta, Sec. 2.3.4), 5x5 median (Sec. 2.1), normals with
// appearance-weighted smoothing and confidence (Sec. 2.4, 2.5), per-pixel
// plane windows (Eq. sampling_range) and surface-normal index jumps
// (Eq. sgm-smooth-sn).  These are bandwidth- or latency-light next to the
// cost volume and the aggregation.
#include <math.h>


#include "../../include/fassmvs.h"
#include "fm_internal.cuh"

namespace fm {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ---------------------------------------------------------------- pyramid
__global__ void pyramid_kernel(const uint8_t* __restrict__ in, int W, int H, int pin,
                               uint8_t* __restrict__ out, int pout)
{
    const int Wo = (W + 1) >> 1, Ho = (H + 1) >> 1;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= Wo || y >= Ho) return;
    const int w[3] = {70, 116, 70};       // 256 * exp(-i^2/2) / sum, rounded (sigma = 1)
    int acc = 0;
#pragma unroll
    for (int j = -1; j <= 1; ++j) {
        const uint8_t* row = in + (size_t)clampi(2 * y + j, 0, H - 1) * pin;
        int hsum = w[0] * row[clampi(2 * x - 1, 0, W - 1)] + w[1] * row[clampi(2 * x, 0, W - 1)] +
                   w[2] * row[clampi(2 * x + 1, 0, W - 1)];
        acc += w[j + 1] * hsum;
    }
    out[(size_t)y * pout + x] = (uint8_t)((acc + 32768) >> 16);
}

// ---------------------------------------------------------------- census
__global__ void census_kernel(const uint8_t* __restrict__ img, int W, int H, int pitch,
                              uint64_t* __restrict__ out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const int c = img[(size_t)y * pitch + x];
    uint64_t bits = 0;
#pragma unroll
    for (int dy = -3; dy <= 3; ++dy) {
        const uint8_t* row = img + (size_t)clampi(y + dy, 0, H - 1) * pitch;
#pragma unroll
        for (int dx = -4; dx <= 4; ++dx) {
            const int k = (dy + 3) * 9 + (dx + 4);
            if (__ldg(row + clampi(x + dx, 0, W - 1)) < c) bits |= 1ull << k;
        }
    }
    out[(size_t)y * W + x] = bits;
}

// ---------------------------------------------------------------- WTA + refinement
// Sbar may be split into nparts partial sums (part_stride elements apart):
// their packed pairs add without carries, as every total stays below 2^16.
__global__ void wta_kernel(const uint16_t* __restrict__ Sbar, const int32_t* __restrict__ lo, int W,
                           int H, int D, int Ds, int G, const float* __restrict__ delta, Intr K, float n0,
                           float n1, float n2, float* __restrict__ depth, int32_t* __restrict__ gwin,
                           int nparts, size_t part_stride, size_t pstride, size_t bstride, int bshift)
{
    const int lane = threadIdx.x & 31;
    const size_t p = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= (size_t)W * H) return;
    const int s0 = lane * 8;
    uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (s0 < D && FM_IN(p * pstride + (size_t)(s0 >> bshift) * bstride + (s0 & ((1 << bshift) - 1)) + 7,
                        (size_t)W * H * Ds, 0x401)) {
        const size_t off = p * pstride + (size_t)(s0 >> bshift) * bstride + (s0 & ((1 << bshift) - 1));
        const uint4* src = reinterpret_cast<const uint4*>(Sbar + off);
        uint4 raw = __ldg(src);
#pragma unroll
        for (int k = 1; k < 8; ++k)
            if (k < nparts) {
                const uint4 t = __ldg(reinterpret_cast<const uint4*>(Sbar + k * part_stride + off));
                raw.x += t.x; raw.y += t.y; raw.z += t.z; raw.w += t.w;
            }
        v[0] = raw.x & 0xFFFF; v[1] = raw.x >> 16; v[2] = raw.y & 0xFFFF; v[3] = raw.y >> 16;
        v[4] = raw.z & 0xFFFF; v[5] = raw.z >> 16; v[6] = raw.w & 0xFFFF; v[7] = raw.w >> 16;
    }
    uint32_t key = 0xFFFFFFFFu;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (s0 + i < D) key = min(key, (v[i] << 8) | (uint32_t)(s0 + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) key = min(key, __shfl_xor_sync(0xFFFFFFFFu, key, o));
    const int s = (int)(key & 255u);
    // neighbour costs c[s-1], c[s+1] from the lanes that hold them
    const int sm = max(s - 1, 0), sp = min(s + 1, D - 1);
    uint32_t vm = 0, vp = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if ((sm & 7) == i) vm = v[i];
        if ((sp & 7) == i) vp = v[i];
    }
    vm = __shfl_sync(0xFFFFFFFFu, vm, sm >> 3);
    vp = __shfl_sync(0xFFFFFFFFu, vp, sp >> 3);
    if (lane != 0) return;
    const int x = (int)(p % W), y = (int)(p / W);
    // a window start with lo + D > G (a caller's map out of contract) stays
    // inside the G-entry table
    const int g = min(max((lo ? lo[p] : 0) + s, 0), G - 1);
    const float x0 = delta[g];
    float xs = x0;
    if (s > 0 && s < D - 1)
        xs = wta_vertex(x0, delta[max(g - 1, 0)], delta[min(g + 1, G - 1)], (float)(key >> 8), (float)vm, (float)vp);
    depth[p] = wta_depth(xs, x, y, K, n0, n1, n2);
    if (gwin) gwin[p] = g;
}

// sum of the aggregation's partial sums (debug capture): out[i] = sum_p Sbar[p * stride + i]
__global__ void sum_parts_kernel(const uint16_t* __restrict__ Sbar, int parts, size_t stride, size_t n,
                                 uint16_t* __restrict__ out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t v = 0;
    for (int p = 0; p < parts; ++p) v += Sbar[(size_t)p * stride + i];
    out[i] = (uint16_t)v;
}

// ---------------------------------------------------------------- volume relayout
// [Ds / 16][np][16] -> [np][Ds], 32 pixels per block of 256 threads: their
// 16-plane blocks are read coalesced (1 KB per block index) into shared
// memory, then written back pixel-major as one contiguous run of 32 x Ds
// planes.  Shared rows are 66 uint4 apart, so that the four pairs of uint4 a
// quarter-warp reads on the way out fall in different banks.
constexpr int kRelPix = 32, kRelRow = 66;
__global__ void __launch_bounds__(256) relayout16_kernel(const uint16_t* __restrict__ src,
                                                         uint16_t* __restrict__ dst, size_t np, int Ds)
{
    __shared__ uint4 sm[kMaxSlots / 16][kRelRow];
    const size_t p0 = (size_t)blockIdx.x * kRelPix;
    const int npx = (int)min((size_t)kRelPix, np - p0);
    const int nb = Ds / 16, per = 2 * nb;      // uint4 per pixel
    for (int i = threadIdx.x; i < nb * 2 * kRelPix; i += blockDim.x) {
        const int b = i / (2 * kRelPix), j = (i >> 1) & (kRelPix - 1), h = i & 1;
        if (j < npx && FM_IN(b, kMaxSlots / 16, 0x402) && FM_IN(((size_t)b * np + p0 + j) * 16 + 15, np * Ds, 0x402))
            sm[b][2 * j + h] = __ldcs(reinterpret_cast<const uint4*>(src + ((size_t)b * np + p0 + j) * 16) + h);
    }
    __syncthreads();
    uint4* d = reinterpret_cast<uint4*>(dst + p0 * (size_t)Ds);
    for (int i = threadIdx.x; i < npx * per; i += blockDim.x) {
        const int j = i / per, k = i - j * per;
        if (FM_IN((p0 + j) * (size_t)Ds + 8 * k + 7, np * Ds, 0x403)) d[i] = sm[k >> 1][2 * j + (k & 1)];
    }
}

// ---------------------------------------------------------------- median 5x5
__global__ void median5_kernel(const float* __restrict__ in, int W, int H, float* __restrict__ out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    float v[25];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i)
            v[5 * j + i] = __ldg(in + (size_t)clampi(y + j - 2, 0, H - 1) * W + clampi(x + i - 2, 0, W - 1));
    // the element of rank 12 (ties broken by position) is the median
    float med = v[0];
#pragma unroll
    for (int i = 0; i < 25; ++i) {
        int rank = 0;
#pragma unroll
        for (int j = 0; j < 25; ++j)
            rank += (v[j] < v[i]) || (v[j] == v[i] && j < i);
        if (rank == 12) med = v[i];
    }
    out[(size_t)y * W + x] = med;
}

// ---------------------------------------------------------------- normals
__device__ __forceinline__ float3 backproject(const float* __restrict__ d, int W, int x, int y, Intr K)
{
    float z = __ldg(d + (size_t)y * W + x);
    return make_float3(z * ((x - K.cx) / K.fx), z * ((y - K.cy) / K.fy), z);
}

__global__ void normal_raw_kernel(const float* __restrict__ depth, int W, int H, Intr K,
                                  float* __restrict__ raw)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    float3 A = backproject(depth, W, min(x + 1, W - 1), y, K);
    float3 B = backproject(depth, W, max(x - 1, 0), y, K);
    float3 C = backproject(depth, W, x, min(y + 1, H - 1), K);
    float3 E = backproject(depth, W, x, max(y - 1, 0), K);
    float3 P = backproject(depth, W, x, y, K);
    float3 h = make_float3(A.x - B.x, A.y - B.y, A.z - B.z);
    float3 v = make_float3(C.x - E.x, C.y - E.y, C.z - E.z);
    float3 c = make_float3(h.y * v.z - h.z * v.y, h.z * v.x - h.x * v.z, h.x * v.y - h.y * v.x);
    float len = sqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
    float* o = raw + 3 * ((size_t)y * W + x);
    if (!(len > 0.0f)) { o[0] = o[1] = o[2] = 0.0f; return; }
    float sgn = (c.x * P.x + c.y * P.y + c.z * P.z) > 0.0f ? -1.0f : 1.0f;
    float inv = sgn / len;
    o[0] = c.x * inv; o[1] = c.y * inv; o[2] = c.z * inv;
}

__global__ void normal_smooth_kernel(const float* __restrict__ raw, const uint8_t* __restrict__ img,
                                     int pitch, int W, int H, int radius, float beta,
                                     float* __restrict__ normal, float np0, float np1, float np2,
                                     float cosr, float* __restrict__ conf)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t p = (size_t)y * W + x;
    const float sigma = (float)radius;
    const float norm = rsqrtf(2.0f * 3.14159265358979f * sigma * sigma);
    const float i2s2 = 1.0f / (2.0f * sigma * sigma);
    const float ib = 1.0f / beta;
    const float Ip = (float)img[(size_t)y * pitch + x];
    float sx = raw[3 * p], sy = raw[3 * p + 1], sz = raw[3 * p + 2];
    for (int j = -radius; j <= radius; ++j) {
        int yy = y + j;
        if (yy < 0 || yy >= H) continue;
        for (int i = -radius; i <= radius; ++i) {
            int xx = x + i;
            if (xx < 0 || xx >= W) continue;
            const size_t q = (size_t)yy * W + xx;
            float dI = fabsf(Ip - (float)img[(size_t)yy * pitch + xx]);
            float w = norm * expf(-(float)(i * i + j * j) * i2s2 - dI * ib);
            sx += w * raw[3 * q];
            sy += w * raw[3 * q + 1];
            sz += w * raw[3 * q + 2];
        }
    }
    float len = sqrtf(sx * sx + sy * sy + sz * sz);
    float inv = len > 0.0f ? 1.0f / len : 0.0f;
    sx *= inv; sy *= inv; sz *= inv;
    normal[3 * p] = sx; normal[3 * p + 1] = sy; normal[3 * p + 2] = sz;
    if (conf) {
        float a = sx * np0 + sy * np1 + sz * np2;
        float b = -np2;
        float c = 0.0f;
        if (a >= cosr && b >= cosr) c = fminf(fmaxf((a * b - cosr) / (1.0f - cosr), 0.0f), 1.0f);
        conf[p] = c;
    }
}

// ---------------------------------------------------------------- window (FP32 decision)
__device__ __forceinline__ float ray_weight(float n0, float n1, float n2, int x, int y, Intr K)
{
    float a = __fdiv_rn(__fsub_rn((float)x, K.cx), K.fx);
    float b = __fdiv_rn(__fsub_rn((float)y, K.cy), K.fy);
    float s = __fadd_rn(__fmul_rn(n0, a), __fmul_rn(n1, b));
    return -__fadd_rn(s, n2);
}

__global__ void window_kernel(const float* __restrict__ dc, int Wc, int Hc, int W, int H, Intr K,
                              float n0, float n1, float n2, float rho0, float drho, int G, int D,
                              int32_t* __restrict__ lo)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    float d = dc[(size_t)min(y >> 1, Hc - 1) * Wc + min(x >> 1, Wc - 1)];
    float w = ray_weight(n0, n1, n2, x, y, K);
    float rho = __fdiv_rn(1.0f, __fmul_rn(d, w));
    float c = __fdiv_rn(__fsub_rn(rho, rho0), drho);
    float fl = floorf(__fadd_rn(c, 0.5f));
    int l;
    if (!(fl > -1.0e9f)) l = 0;
    else if (fl > 1.0e9f) l = G - D;
    else l = (int)fl - D / 2;
    lo[(size_t)y * W + x] = clampi(l, 0, G - D);
}

// ---------------------------------------------------------------- surface-normal jumps (FP32)
// m: the sweep normal; the jump is the change of 1/delta = -1/(m^T X) between
// P and the point where the predecessor ray meets the tangent plane, in the
// oracle's FP32 operation order (for m = (0,0,-1) it is -s1 / (d s0 drho))
__global__ void dsn_kernel(const float* __restrict__ dc, const float* __restrict__ nc, int Wc,
                           int Hc, int W, int H, Intr K, float sw0, float sw1, float sw2, float drho, int dmax,
                           int8_t* __restrict__ dI)
{
    const int kdx[8] = {1, -1, 0, 0, 1, -1, 1, -1};
    const int kdy[8] = {0, 0, 1, -1, 1, -1, -1, 1};
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= W || y >= H) return;
    const size_t pc = (size_t)min(y >> 1, Hc - 1) * Wc + min(x >> 1, Wc - 1);
    const float d = dc[pc];
    const float n0 = nc[3 * pc], n1 = nc[3 * pc + 1], n2 = nc[3 * pc + 2];
    const float a = __fdiv_rn(__fsub_rn((float)x, K.cx), K.fx);
    const float b = __fdiv_rn(__fsub_rn((float)y, K.cy), K.fy);
    const float s0 = __fadd_rn(__fadd_rn(__fmul_rn(n0, a), __fmul_rn(n1, b)), n2);
    const float u0 = __fadd_rn(__fadd_rn(__fmul_rn(sw0, a), __fmul_rn(sw1, b)), sw2);
    const bool nz = (n0 != 0.0f || n1 != 0.0f || n2 != 0.0f);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const float gx = __fdiv_rn((float)kdx[r], K.fx);
        const float gy = __fdiv_rn((float)kdy[r], K.fy);
        const float s1 = __fadd_rn(__fmul_rn(n0, gx), __fmul_rn(n1, gy));
        const float sp = __fsub_rn(s0, s1);
        const float u1 = __fadd_rn(__fmul_rn(sw0, gx), __fmul_rn(sw1, gy));
        const float uq = __fsub_rn(u0, u1);
        int out = 0;
        if (nz && s0 < -1e-6f && sp < -1e-6f && u0 < -1e-6f && uq < -1e-6f && d > 0.0f) {
            const float den = __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(d, s0), u0), uq), drho);
            const float num = __fsub_rn(__fmul_rn(s1, u0), __fmul_rn(s0, u1));
            const float c = __fdiv_rn(num, den);
            float rc = c >= 0.0f ? floorf(__fadd_rn(c, 0.5f)) : -floorf(__fadd_rn(-c, 0.5f));
            rc = fminf(fmaxf(rc, (float)-dmax), (float)dmax);
            out = (int)rc;
        }
        dI[(size_t)r * W * H + (size_t)y * W + x] = (int8_t)out;
    }
}

__global__ void delta_kernel(double rho0, double drho, int G, float* __restrict__ delta)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) delta[g] = (float)(1.0 / (rho0 + (double)g * drho));
}

inline dim3 grid2(int W, int H, dim3 b) { return dim3((W + b.x - 1) / b.x, (H + b.y - 1) / b.y); }

}  // namespace

void launch_pyramid_down(const uint8_t* in, int W, int H, int pin, uint8_t* out, int pout,
                         cudaStream_t st)
{
    dim3 b(32, 8);
    pyramid_kernel<<<grid2((W + 1) / 2, (H + 1) / 2, b), b, 0, st>>>(in, W, H, pin, out, pout);
    count_launch();
}

void launch_census(const uint8_t* img, int W, int H, int pitch, uint64_t* out, cudaStream_t st)
{
    dim3 b(32, 8);
    census_kernel<<<grid2(W, H, b), b, 0, st>>>(img, W, H, pitch, out);
    count_launch();
}

FM_CHECK_TAKE(check_take_stages)

void launch_wta_refine(const uint16_t* Sbar, const int32_t* lo, int W, int H, int D, int Ds, int G,
                       const float* delta, Intr K, const float n[3], float* depth, int32_t* gwin,
                       cudaStream_t st, int nparts, size_t part_stride, size_t pstride, size_t bstride,
                       int bshift)
{
    if (pstride == 0) {
        pstride = (size_t)Ds;
        bstride = 8;
        bshift = 3;
    }
    size_t np = (size_t)W * H;
    int per = 8;
    wta_kernel<<<(unsigned)((np + per - 1) / per), per * 32, 0, st>>>(Sbar, lo, W, H, D, Ds, G, delta, K,
                                                                  n[0], n[1], n[2], depth, gwin, nparts,
                                                                  part_stride, pstride, bstride, bshift);
    count_launch();
}

void launch_relayout16(const uint16_t* src, uint16_t* dst, size_t np, int Ds, cudaStream_t st)
{
    if (np == 0) return;
    relayout16_kernel<<<(unsigned)((np + kRelPix - 1) / kRelPix), 256, 0, st>>>(src, dst, np, Ds);
    count_launch();
}

void launch_sum_parts(const uint16_t* Sbar, int parts, size_t stride, size_t n, uint16_t* out, cudaStream_t st)
{
    if (n == 0) return;
    sum_parts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Sbar, parts, stride, n, out);
    count_launch();
}

void launch_delta_table(double rho0, double drho, int G, float* delta, cudaStream_t st)
{
    delta_kernel<<<(G + 127) / 128, 128, 0, st>>>(rho0, drho, G, delta);
    count_launch();
}

void launch_median5(const float* in, int W, int H, float* out, cudaStream_t st)
{
    dim3 b(32, 8);
    median5_kernel<<<grid2(W, H, b), b, 0, st>>>(in, W, H, out);
    count_launch();
}

void launch_normals(const float* depth, const uint8_t* img, int img_pitch, int W, int H, Intr K,
                    int radius, float beta, float* raw, float* normal, const float npl[3],
                    float rho_deg, float* conf, cudaStream_t st)
{
    dim3 b(32, 8);
    normal_raw_kernel<<<grid2(W, H, b), b, 0, st>>>(depth, W, H, K, raw);
    float cosr = cosf(rho_deg * 3.14159265358979f / 180.0f);
    normal_smooth_kernel<<<grid2(W, H, b), b, 0, st>>>(raw, img, img_pitch, W, H, radius, beta,
                                                       normal, npl[0], npl[1], npl[2], cosr, conf);
    count_launch(2);
}

void launch_window(const float* dc, int Wc, int Hc, int W, int H, Intr K, const float n[3],
                   float rho0, float drho, int G, int D, int32_t* lo, cudaStream_t st)
{
    dim3 b(32, 8);
    window_kernel<<<grid2(W, H, b), b, 0, st>>>(dc, Wc, Hc, W, H, K, n[0], n[1], n[2], rho0, drho, G,
                                                D, lo);
    count_launch();
}

void launch_dsn(const float* dc, const float* nc, int Wc, int Hc, int W, int H, Intr K, const float m[3],
                float drho, int dmax, int8_t* dI, cudaStream_t st)
{
    dim3 b(32, 8);
    dsn_kernel<<<grid2(W, H, b), b, 0, st>>>(dc, nc, Wc, Hc, W, H, K, m[0], m[1], m[2], drho, dmax, dI);
    count_launch();
}

}  // namespace fm

// ---------------------------------------------------------------- no-alloc WTA
// Plane-distance table of fassmvs_wta_refine_noalloc: one static device array
// shared by every call (see the header for the contract).
namespace {
static __device__ __align__(256) float g_noalloc_delta[FASSMVS_NOALLOC_MAX_PLANES];

// device address of the table in the module loaded by the current context.
// Looked up on every call: it is a host-side lookup that allocates nothing,
// and a cached address would dangle once the module is loaded again (after
// cudaDeviceReset, or under another context on the same device).
cudaError_t noalloc_table(float** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_delta);
    if (e != cudaSuccess) return e;
    *out = static_cast<float*>(p);
    return cudaSuccess;
}

fassmvs_status noalloc_fail(fassmvs_status s, const char* msg)
{
    fm::set_error(msg);
    return s;
}
}  // namespace

extern "C" fassmvs_status fassmvs_wta_refine_noalloc(const uint16_t* Sbar, const int32_t* lo, int W, int H,
                                                     int D, int Ds, const double K[9], const double n[3],
                                                     double rho0, double drho, int G, float* depth,
                                                     int32_t* gwin, void* stream)
{
    if (!Sbar || !K || !n || !depth || W < 1 || H < 1)
        return noalloc_fail(FASSMVS_EINVAL, "bad WTA arguments");
    if (D < 1 || D > fm::kMaxSlots || Ds < D || (Ds & 7) || G < D)
        return noalloc_fail(FASSMVS_EINVAL, "bad D / Ds / G");
    if (G > FASSMVS_NOALLOC_MAX_PLANES)
        return noalloc_fail(FASSMVS_EINVAL, "G exceeds the static plane table of the no-alloc entry point (4096)");
    if (reinterpret_cast<uintptr_t>(Sbar) & 15)
        return noalloc_fail(FASSMVS_EINVAL, "volume must be 16-byte aligned");
    float* table = nullptr;
    cudaError_t e = noalloc_table(&table);
    if (e != cudaSuccess) return noalloc_fail(FASSMVS_ECUDA, cudaGetErrorString(e));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    fm::launch_delta_table(rho0, drho, G, table, st);
    float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
    fm::Intr ki{(float)K[0], (float)K[4], (float)K[2], (float)K[5]};
    fm::launch_wta_refine(Sbar, lo, W, H, D, Ds, G, table, ki, nf, depth, gwin, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FASSMVS_ECUDA, cudaGetErrorString(e));
    return FASSMVS_OK;
}
