// Post-filters of Sec. 2.6 for sm_103a: the difference-of-Gaussian texture
// mask (Alg. 3) and the geometric consistency check by mutual reprojection
// (Alg. 4).
//
// The DoG mask is integer work: a 7x7 fixed-point Gaussian (weights summing
// to 256 per axis) and threshold in one shared-memory tile kernel, speckle
// removal by connected-component labelling (lock-free union-find: a root is
// linked under the smaller root with atomicMin; parents only ever decrease, so
// every walk ends; path compression also writes by atomicMin), component sizes
// by atomicAdd, a 3x3 dilation.  The result is exactly the oracle's.
// The reprojection check is FP64 with every operation explicitly rounded in
// the oracle's order (the hit decision is an integer one).
#include "fm_internal.cuh"

namespace fm {

namespace {

constexpr int TX = 32, TY = 8;
// bounded walks: parents strictly decrease, so a walk is at most the image
// size long; a walk that reaches the cap flags an error instead of spinning
constexpr int kWalkCap = 1 << 26;

__global__ void dog_threshold_kernel(const uint8_t* __restrict__ img, int W, int H, int pitch, const DogWeights dw,
                                     uint8_t* __restrict__ mask)
{
    __shared__ uint8_t tile[TY + 6][TX + 6];
    __shared__ int32_t hs[TY + 6][TX];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    for (int i = threadIdx.y * TX + threadIdx.x; i < (TY + 6) * (TX + 6); i += TX * TY) {
        const int r = i / (TX + 6), c = i % (TX + 6);
        const int y = min(max(y0 + r - 3, 0), H - 1), x = min(max(x0 + c - 3, 0), W - 1);
        tile[r][c] = img[(size_t)y * pitch + x];
    }
    __syncthreads();
    for (int i = threadIdx.y * TX + threadIdx.x; i < (TY + 6) * TX; i += TX * TY) {
        const int r = i / TX, c = i % TX;
        int32_t a = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) a += dw.w[k] * (int32_t)tile[r][c + k];
        hs[r][c] = a;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= W || y >= H) return;
    int64_t a = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) a += (int64_t)dw.w[k] * hs[threadIdx.y + k][threadIdx.x];
    const int64_t dog = ((int64_t)tile[threadIdx.y + 3][threadIdx.x + 3] << 16) - a;
    mask[(size_t)y * W + x] = (dog > 32768 || dog < -32768) ? 1 : 0;
}

__device__ __forceinline__ int find_root(int* parent, int p, int* err)
{
    int r = p;
    for (int it = 0; it < kWalkCap; ++it) {
        const int q = *(volatile int*)&parent[r];
        if (q == r) {
            // compress: point p at the root (values only decrease)
            if (p != r) atomicMin(&parent[p], r);
            return r;
        }
        r = q;
    }
    atomicExch(err, 1);
    return r;
}

__device__ __forceinline__ void unite(int* parent, int a, int b, int* err)
{
    for (int it = 0; it < kWalkCap; ++it) {
        a = find_root(parent, a, err);
        b = find_root(parent, b, err);
        if (a == b) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(&parent[a], b);
        if (old == a) return;              // a was a root: linked under b
        a = old;                           // a was linked meanwhile: unite its new parent
    }
    atomicExch(err, 1);
}

__global__ void ccl_init_kernel(const uint8_t* __restrict__ m, int n, uint8_t val, int* parent, int* size)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    parent[p] = m[p] == val ? p : -1;
    size[p] = 0;
}

__global__ void ccl_merge_kernel(const uint8_t* __restrict__ m, int W, int H, uint8_t val, int* parent, int* err)
{
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= W || y >= H) return;
    const int p = y * W + x;
    if (m[p] != val) return;
    if (x + 1 < W && m[p + 1] == val) unite(parent, p, p + 1, err);
    if (y + 1 < H && m[p + W] == val) unite(parent, p, p + W, err);
}

__global__ void ccl_count_kernel(const uint8_t* __restrict__ m, int n, uint8_t val, int* parent, int* size, int* err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || m[p] != val) return;
    const int r = find_root(parent, p, err);
    atomicAdd(&size[r], 1);
}

__global__ void ccl_apply_kernel(uint8_t* m, int n, uint8_t val, int minsize, int* parent, const int* size, int* err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || m[p] != val) return;
    const int r = find_root(parent, p, err);
    if (size[r] < minsize) m[p] = (uint8_t)(1 - val);
}

__global__ void dilate3_kernel(const uint8_t* __restrict__ in, int W, int H, uint8_t* __restrict__ out)
{
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= W || y >= H) return;
    uint8_t v = 0;
    for (int j = max(y - 1, 0); j <= min(y + 1, H - 1); ++j)
        for (int i = max(x - 1, 0); i <= min(x + 1, W - 1); ++i) v |= in[(size_t)j * W + i];
    out[(size_t)y * W + x] = v;
}

__global__ void apply_mask_kernel(const uint8_t* __restrict__ m, int n, float* depth, float* normal, float* conf)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || m[p]) return;
    depth[p] = 0.0f;
    normal[3 * p] = normal[3 * p + 1] = normal[3 * p + 2] = 0.0f;
    conf[p] = 0.0f;
}

__global__ void geo_kernel(const GeoArgs g, float* depth, float* normal, float* conf, uint8_t* hits_out)
{
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= g.W || y >= g.H) return;
    const size_t p = (size_t)y * g.W + x;
    const double fx = g.fx, fy = g.fy, cx = g.cx, cy = g.cy;
    int h = 0;
    const double d = depth[p];
    if (d > 0.0) {
        const double X0 = __dmul_rn(__ddiv_rn(__dsub_rn((double)x, cx), fx), d);
        const double X1 = __dmul_rn(__ddiv_rn(__dsub_rn((double)y, cy), fy), d);
        const double X2 = d;
        for (int k = 0; k < g.n; ++k) {
            const double* R = g.R[k];
            const double* t = g.t[k];
            const double Y0 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[0], X0), __dmul_rn(R[1], X1)), __dmul_rn(R[2], X2)), t[0]);
            const double Y1 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[3], X0), __dmul_rn(R[4], X1)), __dmul_rn(R[5], X2)), t[1]);
            const double Y2 = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[6], X0), __dmul_rn(R[7], X1)), __dmul_rn(R[8], X2)), t[2]);
            if (!(Y2 > 0.0)) continue;
            const double u = __dadd_rn(__ddiv_rn(__dmul_rn(fx, Y0), Y2), cx);
            const double v = __dadd_rn(__ddiv_rn(__dmul_rn(fy, Y1), Y2), cy);
            const double ru = floor(__dadd_rn(u, 0.5)), rv = floor(__dadd_rn(v, 0.5));
            if (!(ru >= 0.0 && ru <= g.W - 1 && rv >= 0.0 && rv <= g.H - 1)) continue;
            const double e = g.dk[k][(size_t)rv * g.W + (size_t)ru];
            if (!(e > 0.0)) continue;
            const double Z0 = __dsub_rn(__dmul_rn(__ddiv_rn(__dsub_rn(u, cx), fx), e), t[0]);
            const double Z1 = __dsub_rn(__dmul_rn(__ddiv_rn(__dsub_rn(v, cy), fy), e), t[1]);
            const double Z2 = __dsub_rn(e, t[2]);
            const double B0 = __dadd_rn(__dadd_rn(__dmul_rn(R[0], Z0), __dmul_rn(R[3], Z1)), __dmul_rn(R[6], Z2));
            const double B1 = __dadd_rn(__dadd_rn(__dmul_rn(R[1], Z0), __dmul_rn(R[4], Z1)), __dmul_rn(R[7], Z2));
            const double B2 = __dadd_rn(__dadd_rn(__dmul_rn(R[2], Z0), __dmul_rn(R[5], Z1)), __dmul_rn(R[8], Z2));
            if (!(B2 > 0.0)) continue;
            const double du = __dsub_rn(__dadd_rn(__ddiv_rn(__dmul_rn(fx, B0), B2), cx), (double)x);
            const double dv = __dsub_rn(__dadd_rn(__ddiv_rn(__dmul_rn(fy, B1), B2), cy), (double)y);
            if (__dsqrt_rn(__dadd_rn(__dmul_rn(du, du), __dmul_rn(dv, dv))) < g.eta_r) ++h;
        }
    }
    if (hits_out) hits_out[p] = (uint8_t)h;
    if (h < g.eta_h) {
        depth[p] = 0.0f;
        if (normal) normal[3 * p] = normal[3 * p + 1] = normal[3 * p + 2] = 0.0f;
        if (conf) conf[p] = 0.0f;
    }
}

dim3 grid2d(int W, int H) { return dim3((W + TX - 1) / TX, (H + TY - 1) / TY); }

void speckle(uint8_t* m, int W, int H, uint8_t val, int minsize, int* parent, int* size, int* err, cudaStream_t st)
{
    const int n = W * H, b = 256, nb = (n + b - 1) / b;
    ccl_init_kernel<<<nb, b, 0, st>>>(m, n, val, parent, size);
    ccl_merge_kernel<<<grid2d(W, H), dim3(TX, TY), 0, st>>>(m, W, H, val, parent, err);
    ccl_count_kernel<<<nb, b, 0, st>>>(m, n, val, parent, size, err);
    ccl_apply_kernel<<<nb, b, 0, st>>>(m, n, val, minsize, parent, size, err);
    count_launch(4);
}

}  // namespace

void launch_dog_mask(const uint8_t* img, int W, int H, int pitch, const DogWeights& dw, uint8_t* mask, uint8_t* tmp,
                     int* parent, int* size, int* err, cudaStream_t st)
{
    dog_threshold_kernel<<<grid2d(W, H), dim3(TX, TY), 0, st>>>(img, W, H, pitch, dw, mask);
    count_launch();
    speckle(mask, W, H, 1, 7, parent, size, err, st);
    dilate3_kernel<<<grid2d(W, H), dim3(TX, TY), 0, st>>>(mask, W, H, tmp);
    count_launch();
    speckle(tmp, W, H, 0, 21, parent, size, err, st);
    cudaMemcpyAsync(mask, tmp, (size_t)W * H, cudaMemcpyDeviceToDevice, st);
}

void launch_apply_mask(const uint8_t* mask, int W, int H, float* depth, float* normal, float* conf, cudaStream_t st)
{
    const int n = W * H;
    apply_mask_kernel<<<(n + 255) / 256, 256, 0, st>>>(mask, n, depth, normal, conf);
    count_launch();
}

void launch_geo_filter(const GeoArgs& g, float* depth, float* normal, float* conf, uint8_t* hits, cudaStream_t st)
{
    geo_kernel<<<grid2d(g.W, g.H), dim3(TX, TY), 0, st>>>(g, depth, normal, conf, hits);
    count_launch();
}

}  // namespace fm
