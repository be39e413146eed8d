/*
 * FaSS-MVS CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct restatement of the hot path of FaSS-MVS
 * (Ruf, Weinmann, Hinz; arXiv 2112.00821) in C with FP64 arithmetic.  It is
 * used by the test-suite, by the smoke check and by the benchmark's CPU
 * baseline leg, and by nothing else: the product path never links or calls
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library.  Each function names the paper passage it restates.  Where the
 * paper is silent, the reading taken is stated next to the code.
 *
 * Data layouts (row-major):
 *   images          uint8  [H][W]
 *   census          uint64 [H][W]
 *   cost volumes    uint16 [H][W][Ds]   (slot s of pixel p is plane lo_p + s;
 *                                        Ds >= D is the slot stride)
 *   window offsets  int32  [H][W]       (lo_p; NULL means lo_p = 0)
 *   depth           float  [H][W]
 *   normals         float  [H][W][3]
 *   dI (sn)         int8   [8][H][W]
 *
 * Precision: FP64 everywhere, except the two places where a floating-point
 * value decides a small integer that both implementations must agree on
 * (the per-pixel plane window and the surface-normal index jump); there the
 * decision is taken in FP32 with every operation spelled out (no contraction,
 * IEEE single rounding), because that is the precision the GPU takes it in.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: Gaussian pyramid. 3x3 Gaussian with sigma = 1, then scaling by  */
/* 0.5 in both directions; K is adjusted by halving f and the principal     */
/* point.  Reading: the kernel is the separable [w0 w1 w0] obtained by       */
/* rounding 256 * g / sum(g) with g = exp(-x^2 / 2), x = -1, 0, 1; the output */
/* pixel (x, y) is the blurred input at (2x, 2y) with clamp-to-edge, rounded */
/* half up after dividing by 2^16; the output size is ceil(W/2) x ceil(H/2). */
/* ------------------------------------------------------------------------ */
/* Thread count of the parallel loops over independent pixels and lines
   (timing only: no result depends on it).  n >= 1 sets it, 0 leaves it;
   returns the count in force. */
OR_EXPORT int or_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

OR_EXPORT void or_pyr_weights(int32_t w[3])
{
    double g1 = exp(-0.5), g0 = 1.0;
    double s = g0 + 2.0 * g1;
    w[0] = (int32_t)floor(256.0 * g1 / s + 0.5);
    w[1] = (int32_t)floor(256.0 * g0 / s + 0.5);
    w[2] = w[0];
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

OR_EXPORT void or_pyramid_down(const uint8_t* in, int W, int H, uint8_t* out)
{
    int32_t w[3];
    or_pyr_weights(w);
    int Wo = (W + 1) / 2, Ho = (H + 1) / 2;
    for (int y = 0; y < Ho; ++y)
        for (int x = 0; x < Wo; ++x) {
            int64_t acc = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) {
                    int xx = clampi(2 * x + i, 0, W - 1), yy = clampi(2 * y + j, 0, H - 1);
                    acc += (int64_t)w[i + 1] * w[j + 1] * in[(size_t)yy * W + xx];
                }
            out[(size_t)y * Wo + x] = (uint8_t)((acc + 32768) >> 16);
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.1 and Sec. 3.4: census transform (Zabih & Woodfill) over a 9x7   */
/* support region, which fits one 64-bit word.  Reading: bit k of the string */
/* for pixel p is [I(q) < I(p)] with q = p + (dx, dy), dx in -4..4, dy in     */
/* -3..3, k = (dy + 3) * 9 + (dx + 4) (row-major); the centre bit (k = 31)   */
/* is always 0, so the Hamming distance of two strings is at most 62.        */
/* Taps outside the image use clamp-to-edge.                                 */
/* ------------------------------------------------------------------------ */
OR_EXPORT void or_census_u8(const uint8_t* img, int W, int H, uint64_t* out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int c = img[(size_t)y * W + x];
            uint64_t bits = 0;
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -4; dx <= 4; ++dx) {
                    int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
                    int k = (dy + 3) * 9 + (dx + 4);
                    if (img[(size_t)yy * W + xx] < c) bits |= (uint64_t)1 << k;
                }
            out[(size_t)y * W + x] = bits;
        }
}

/* census over a warped image of real values (the warped neighbour patches),
   whose rows ya .. are stored in img */
static uint64_t census_f64_at(const double* img, int W, int H, int ya, int x, int y)
{
    double c = img[(size_t)(y - ya) * W + x];
    uint64_t bits = 0;
    for (int dy = -3; dy <= 3; ++dy)
        for (int dx = -4; dx <= 4; ++dx) {
            int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
            int k = (dy + 3) * 9 + (dx + 4);
            if (img[(size_t)(yy - ya) * W + xx] < c) bits |= (uint64_t)1 << k;
        }
    return bits;
}

static int popcount64(uint64_t v)
{
    int n = 0;
    while (v) { n += (int)(v & 1u); v >>= 1; }
    return n;
}

OR_EXPORT int or_hamming(uint64_t a, uint64_t b) { return popcount64(a ^ b); }

/* ------------------------------------------------------------------------ */
/* Sec. 2.2, Eq. homography: the plane Pi = (n, delta) maps reference pixels */
/* to neighbour pixels by H = K (R - t n^T / delta) K^-1, where X_k = R X +  */
/* t and the plane is n^T X + delta = 0 in the reference frame (for the      */
/* fronto-parallel n = (0,0,-1), delta is the depth).  The typeset equation  */
/* places delta under R - t n^T; the plane-induced homography of Hartley &   */
/* Zisserman that the paper cites divides only t n^T by delta.              */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double* A, const double* B, double* C)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof(T));
}

static void mat3_inv(const double* A, double* B)
{
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    B[0] = c00 / det;
    B[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    B[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    B[3] = c01 / det;
    B[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    B[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    B[6] = c02 / det;
    B[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    B[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}

OR_EXPORT void or_homography(const double K[9], const double R[9], const double t[3],
                             const double n[3], double delta, double Hm[9])
{
    double M[9], Ki[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] - t[i] * n[j] / delta;
    mat3_inv(K, Ki);
    mat3_mul(K, M, M);
    mat3_mul(M, Ki, Hm);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 (patch warping step): bringing the neighbour patch around H p into */
/* the reference view is the same as sampling I_k at H q for every q of the */
/* reference support window.  Reading of the sampling (the paper does not   */
/* fix it): the position (u, v) = H q is taken in FP64 without rounding,    */
/* clamped to the image (clamp-to-edge), and the image is interpolated      */
/* bilinearly in lerp form from the 2x2 pixels around it:                   */
/*   top = I00 + a (I01 - I00), bottom = I10 + a (I11 - I10),                */
/*   value = top + b (bottom - top),                                         */
/* with a, b the offsets of the clamped position from the top-left pixel    */
/* (equal corners give that grey level exactly).  The value is a real      */
/* number, not rounded.  A point behind the neighbour camera (homogeneous   */
/* w <= 0) is treated as lying at (-inf, -inf).                             */
/* ------------------------------------------------------------------------ */
/* position of reference pixel (x, y) in the neighbour; returns 0 when the
   point is behind the neighbour camera */
static int warp_pos(const double* Hm, int x, int y, double* u, double* v)
{
    double a = Hm[0] * x + Hm[1] * y + Hm[2];
    double b = Hm[3] * x + Hm[4] * y + Hm[5];
    double w = Hm[6] * x + Hm[7] * y + Hm[8];
    if (!(w > 0.0)) { *u = -INFINITY; *v = -INFINITY; return 0; }
    *u = a / w;
    *v = b / w;
    return 1;
}

static double bilinear(const uint8_t* img, int W, int H, double u, double v)
{
    double cu = u > 0.0 ? (u < (double)(W - 1) ? u : (double)(W - 1)) : 0.0;   /* NaN -> 0 */
    double cv = v > 0.0 ? (v < (double)(H - 1) ? v : (double)(H - 1)) : 0.0;
    int iu = (int)floor(cu), iv = (int)floor(cv);
    if (iu > W - 2) iu = W - 2;
    if (iv > H - 2) iv = H - 2;
    double a = cu - iu, b = cv - iv;
    const uint8_t* r0 = img + (size_t)iv * W + iu;
    const uint8_t* r1 = r0 + W;
    double top = r0[0] + a * ((double)r0[1] - r0[0]);
    double bot = r1[0] + a * ((double)r1[1] - r1[0]);
    return top + b * (bot - top);
}

/* value of the warped neighbour at reference pixel (x, y); *valid tells
   whether the (unclamped) position lies on the image grid */
OR_EXPORT double or_warp_sample(const uint8_t* img, int W, int H, const double Hm[9], int x, int y,
                                int32_t* valid)
{
    double u, v;
    int front = warp_pos(Hm, x, y, &u, &v);
    if (valid) *valid = front && u >= 0.0 && u <= (double)(W - 1) && v >= 0.0 && v <= (double)(H - 1);
    return bilinear(img, W, H, u, v);
}

OR_EXPORT void or_warp_image(const uint8_t* img, int W, int H, const double Hm[9], double* out,
                             uint8_t* valid)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int32_t v;
            out[(size_t)y * W + x] = or_warp_sample(img, W, H, Hm, x, y, &v);
            if (valid) valid[(size_t)y * W + x] = (uint8_t)v;
        }
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 and the occlusion handling of Kang et al.: per pixel and plane,    */
/* s^L = sum of the costs of the views left of the reference (k < ref),      */
/* s^R = sum over the views to the right, S = min(s^L, s^R).  Readings:      */
/* (a) a view whose centre sample leaves the image contributes the maximal   */
/* census cost 62; (b) with unequal subsets each sum is rescaled to          */
/* n_max = max(n_L, n_R) images with integer round-half-up,                   */
/* s_hat = (s * n_max + n / 2) / n; an empty side is ignored.                */
/* ------------------------------------------------------------------------ */
OR_EXPORT uint16_t or_lr_combine(uint32_t sL, int nL, uint32_t sR, int nR)
{
    int nmax = nL > nR ? nL : nR;
    uint32_t a = 0xFFFFFFFFu, b = 0xFFFFFFFFu;
    if (nL > 0) a = (sL * (uint32_t)nmax + (uint32_t)(nL / 2)) / (uint32_t)nL;
    if (nR > 0) b = (sR * (uint32_t)nmax + (uint32_t)(nR / 2)) / (uint32_t)nR;
    return (uint16_t)(a < b ? a : b);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.1, the NCC alternative to the census (Sec. 3.4 selects a 5x5     */
/* support region; the maximal cost is normalised to 255).  Reading: the     */
/* correlation coefficient of the reference window a (grey levels) and the   */
/* warped window b (real values, as for the census),                         */
/* ncc = sum (a - mean a)(b - mean b) / sqrt(sum (a - mean a)^2 sum (b - mean b)^2), */
/* negated, truncated at zero correlation and scaled:                        */
/* C = round_half_up(255 (1 - max(ncc, 0))); a flat window (zero variance)   */
/* costs 255, as does an invalid view.                                       */
/* ------------------------------------------------------------------------ */
OR_EXPORT int or_ncc_window(const double a[25], const double b[25])
{
    double ma = 0.0, mb = 0.0;
    for (int i = 0; i < 25; ++i) { ma += a[i]; mb += b[i]; }
    ma /= 25.0;
    mb /= 25.0;
    double cov = 0.0, va = 0.0, vb = 0.0;
    for (int i = 0; i < 25; ++i) {
        cov += (a[i] - ma) * (b[i] - mb);
        va += (a[i] - ma) * (a[i] - ma);
        vb += (b[i] - mb) * (b[i] - mb);
    }
    if (!(va > 0.0) || !(vb > 0.0)) return 255;
    double ncc = cov / sqrt(va * vb);
    if (ncc < 0.0) ncc = 0.0;
    int c = (int)floor(255.0 * (1.0 - ncc) + 0.5);
    return c < 0 ? 0 : (c > 255 ? 255 : c);
}

/* NCC cost of pixel (x, y): 5x5 windows with clamp-to-edge in the reference
   grid over the reference image and the warped image, whose rows ya .. are
   stored in wimg. */
static int ncc_at(const uint8_t* ref, const double* wimg, int W, int H, int ya, int x, int y)
{
    double a[25], b[25];
    int i = 0;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx, ++i) {
            const int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
            a[i] = ref[(size_t)yy * W + xx];
            b[i] = wimg[(size_t)(yy - ya) * W + xx];
        }
    return or_ncc_window(a, b);
}

/* Plane list of a level (Sec. 2.2.3 and Sec. 2.1): planes uniform in inverse
   depth, 1/delta_g = rho0 + g * drho, g = 0 the farthest. */
static double plane_delta(double rho0, double drho, int g) { return 1.0 / (rho0 + g * drho); }

/*
 * Cost volume of one pyramid level (Alg. 1), rows y0 .. y1 - 1 of the
 * reference.  For every neighbour view and every plane g of the level list
 * needed by some pixel, the neighbour image is warped into the reference view
 * (the rows the band's windows reach), its census is taken at the pixels
 * whose window [lo_p, lo_p + D) contains g, and the Hamming distance to the
 * reference census is accumulated into the left or right subset sum (cost
 * 0), or the NCC cost of the 5x5 windows (cost 1) is.
 * R: V x 9 (row-major), t: V x 3, side: -1 left / +1 right; lo: [H][W] of the
 * whole image (or NULL); S: [y1 - y0][W][Ds].
 */
OR_EXPORT int or_cost_band(const uint8_t* ref, const uint8_t* const* nbrs, int V,
                           const int8_t* side, int W, int H, const double K[9],
                           const double* R, const double* t, const double n[3],
                           double rho0, double drho, int G, const int32_t* lo,
                           int D, int Ds, int cost, int y0, int y1, uint16_t* S)
{
    if (W < 2 || H < 2 || D < 1 || Ds < D || G < D || y0 < 0 || y1 > H || y0 >= y1) return -1;
    const int ya = y0 - 3 < 0 ? 0 : y0 - 3, yb = y1 + 3 > H ? H : y1 + 3;   /* warped rows */
    const size_t nb = (size_t)W * (y1 - y0), nw = (size_t)W * (yb - ya);
    uint64_t* cref = (uint64_t*)malloc((size_t)W * H * sizeof(uint64_t));
    uint32_t* sL = (uint32_t*)calloc(nb * D, sizeof(uint32_t));
    uint32_t* sR = (uint32_t*)calloc(nb * D, sizeof(uint32_t));
    int nL = 0, nR = 0;
    for (int k = 0; k < V; ++k) { if (side[k] < 0) ++nL; else ++nR; }
    or_census_u8(ref, W, H, cref);
    int gmin = G, gmax = -1;
    for (int y = y0; y < y1; ++y)
        for (int x = 0; x < W; ++x) {
            int l = lo ? lo[(size_t)y * W + x] : 0;
            if (l < gmin) gmin = l;
            if (l + D - 1 > gmax) gmax = l + D - 1;
        }
    for (int k = 0; k < V; ++k) {
#pragma omp parallel
        {
            double* wimg = (double*)malloc(nw * sizeof(double));
            uint8_t* wval = (uint8_t*)malloc(nw);
            double Hm[9];
#pragma omp for schedule(dynamic, 1)
            for (int g = gmin; g <= gmax; ++g) {
                or_homography(K, R + 9 * k, t + 3 * k, n, plane_delta(rho0, drho, g), Hm);
                for (int y = ya; y < yb; ++y)
                    for (int x = 0; x < W; ++x) {
                        int32_t v;
                        wimg[(size_t)(y - ya) * W + x] = or_warp_sample(nbrs[k], W, H, Hm, x, y, &v);
                        wval[(size_t)(y - ya) * W + x] = (uint8_t)v;
                    }
                for (int y = y0; y < y1; ++y)
                    for (int x = 0; x < W; ++x) {
                        size_t p = (size_t)y * W + x, pb = (size_t)(y - y0) * W + x;
                        int s = g - (lo ? lo[p] : 0);
                        if (s < 0 || s >= D) continue;
                        int h = cost ? 255 : 62;
                        if (wval[(size_t)(y - ya) * W + x])
                            h = cost ? ncc_at(ref, wimg, W, H, ya, x, y)
                                     : or_hamming(cref[p], census_f64_at(wimg, W, H, ya, x, y));
                        if (side[k] < 0) sL[pb * D + s] += (uint32_t)h;
                        else sR[pb * D + s] += (uint32_t)h;
                    }
            }
            free(wimg);
            free(wval);
        }
    }
    for (size_t p = 0; p < nb; ++p)
        for (int s = 0; s < Ds; ++s)
            S[p * Ds + s] = s < D ? or_lr_combine(sL[p * D + s], nL, sR[p * D + s], nR) : 0;
    free(cref);
    free(sL);
    free(sR);
    return 0;
}

/* the whole image */
OR_EXPORT int or_cost_volume(const uint8_t* ref, const uint8_t* const* nbrs, int V,
                             const int8_t* side, int W, int H, const double K[9],
                             const double* R, const double* t, const double n[3],
                             double rho0, double drho, int G, const int32_t* lo,
                             int D, int Ds, int cost, uint16_t* S)
{
    return or_cost_band(ref, nbrs, V, side, W, H, K, R, t, n, rho0, drho, G, lo, D, Ds, cost, 0, H, S);
}

/* The same cost for a list of individual voxels (pixel (x, y), plane g of
   the level list), each computed on its own from the 9x7 window of warped
   samples around the pixel -- used to check full-size volumes by sampling. */
OR_EXPORT void or_cost_at(const uint8_t* ref, const uint8_t* const* nbrs, int V, const int8_t* side,
                          int W, int H, const double K[9], const double* R, const double* t,
                          const double n[3], double rho0, double drho, int npts, const int32_t* xs,
                          const int32_t* ys, const int32_t* gs, int cost, uint16_t* out)
{
    int nL = 0, nR = 0;
    for (int k = 0; k < V; ++k) { if (side[k] < 0) ++nL; else ++nR; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < npts; ++i) {
        int x = xs[i], y = ys[i];
        uint64_t cref = 0;
        int c0 = ref[(size_t)y * W + x];
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -4; dx <= 4; ++dx) {
                int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
                if (ref[(size_t)yy * W + xx] < c0) cref |= (uint64_t)1 << ((dy + 3) * 9 + dx + 4);
            }
        uint32_t sL = 0, sR = 0;
        double Hm[9];
        for (int k = 0; k < V; ++k) {
            or_homography(K, R + 9 * k, t + 3 * k, n, plane_delta(rho0, drho, gs[i]), Hm);
            int32_t valid;
            double cen = or_warp_sample(nbrs[k], W, H, Hm, x, y, &valid);
            int h = cost ? 255 : 62;
            if (valid && cost) {
                double a[25], b[25];
                int i = 0;
                for (int dy = -2; dy <= 2; ++dy)
                    for (int dx = -2; dx <= 2; ++dx, ++i) {
                        int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
                        a[i] = ref[(size_t)yy * W + xx];
                        b[i] = or_warp_sample(nbrs[k], W, H, Hm, xx, yy, NULL);
                    }
                h = or_ncc_window(a, b);
            } else if (valid) {
                uint64_t bits = 0;
                for (int dy = -3; dy <= 3; ++dy)
                    for (int dx = -4; dx <= 4; ++dx) {
                        int xx = clampi(x + dx, 0, W - 1), yy = clampi(y + dy, 0, H - 1);
                        if (or_warp_sample(nbrs[k], W, H, Hm, xx, yy, NULL) < cen)
                            bits |= (uint64_t)1 << ((dy + 3) * 9 + dx + 4);
                    }
                h = or_hamming(cref, bits);
            }
            if (side[k] < 0) sL += (uint32_t)h; else sR += (uint32_t)h;
        }
        out[i] = or_lr_combine(sL, nL, sR, nR);
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3.3, Eq. p2-grad: phi2 = phi1 (1 + alpha exp(-dI / beta)), with    */
/* the penalties multiplied by the number of images per subset.  Reading:    */
/* phi1 is given already multiplied; the table is rounded half up.           */
/* ------------------------------------------------------------------------ */
OR_EXPORT void or_p2_table(int p1, double alpha, double beta, uint16_t lut[256])
{
    for (int d = 0; d < 256; ++d)
        lut[d] = (uint16_t)floor((double)p1 * (1.0 + alpha * exp(-(double)d / beta)) + 0.5);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.3: SGM path aggregation adapted to plane hypotheses.              */
/*   Eq. xsgm:          L_r(p,Pi) = S(p,Pi) + min_Pi' (L_r(p-r,Pi') + V)     */
/*   Eq. sgm-smooth-fp: V = 0 / phi1 / phi2 for index difference 0 / 1 / >1 */
/*   Eq. sgm-smooth-sn, Eq. sgm-smooth-pg: V(Pi + di, Pi')                    */
/*   Eq. sgm-aggr:      S_bar = sum_r L_r                                     */
/* Readings: the standard normalised form (subtract M = min_k L_r(p-r, k),   */
/* which leaves the arg-min of S_bar unchanged); the predecessor of p on     */
/* path r is p - r; the first pixel of a path has L_r = S; hypotheses      */
/* outside the predecessor's window count as +infinity; phi2 is raised to   */
/* phi1 when smaller.  With windows, slot s of p is plane lo_p + s, and the  */
/* zero-cost transition is to plane lo_p + s + di, i.e. slot                 */
/* s + lo_p - lo_{p-r} + di of the predecessor.                              */
/* Path order (r index): 0:(1,0) 1:(-1,0) 2:(0,1) 3:(0,-1) 4:(1,1) 5:(-1,-1) */
/* 6:(1,-1) 7:(-1,1); four paths use r = 0..3.                               */
/* di for sn comes from dI[r][y][x]; for pg it is g(p-2r) - g(p-r) where     */
/* g(x) = lo_x + argmin_s L_r(x, s) (lowest s on ties), 0 for the first two  */
/* pixels of a path, clamped to +-dmax.                                      */
/* ------------------------------------------------------------------------ */
static const int OR_DX[8] = {1, -1, 0, 0, 1, -1, 1, -1};
static const int OR_DY[8] = {0, 0, 1, -1, 1, -1, -1, 1};

OR_EXPORT void or_path_dir(int r, int* dx, int* dy) { *dx = OR_DX[r]; *dy = OR_DY[r]; }

typedef struct {
    int32_t W, H, D, Ds, G;
    int32_t paths;       /* 8 or 4 */
    int32_t variant;     /* 0 plane-wise, 1 surface normal, 2 path gradient */
    int32_t p1;          /* phi1 (already multiplied) */
    int32_t p2;          /* phi2 when lut == NULL */
    int32_t dmax;
} or_sgm_params;

/* One aggregation step (Eq. xsgm, normalised). Lp: predecessor costs (D),
   sh: slot shift, S: data costs of p (D), out: L_r(p, .) */
static void sgm_step(const uint32_t* Lp, int D, int sh, int P1, int P2, const uint16_t* S,
                     uint32_t* out)
{
    uint32_t M = 0xFFFFFFFFu;
    for (int k = 0; k < D; ++k) if (Lp[k] < M) M = Lp[k];
    for (int s = 0; s < D; ++s) {
        int q = s + sh;
        uint32_t best = M + (uint32_t)P2;
        if (q >= 0 && q < D && Lp[q] < best) best = Lp[q];
        if (q - 1 >= 0 && q - 1 < D && Lp[q - 1] + (uint32_t)P1 < best) best = Lp[q - 1] + (uint32_t)P1;
        if (q + 1 >= 0 && q + 1 < D && Lp[q + 1] + (uint32_t)P1 < best) best = Lp[q + 1] + (uint32_t)P1;
        out[s] = (uint32_t)S[s] + best - M;
    }
}

static int argmin_u32(const uint32_t* v, int D)
{
    int a = 0;
    for (int k = 1; k < D; ++k) if (v[k] < v[a]) a = k;
    return a;
}

/* Aggregate one path direction; adds L_r into acc (uint32, H*W*D) and, when
   Lout != NULL, also stores L_r itself. */
static void sgm_direction(const uint16_t* S, const int32_t* lo, const int8_t* dI,
                          const uint8_t* img, const uint16_t* lut, const or_sgm_params* P,
                          int r, uint32_t* acc, uint32_t* Lout)
{
    int W = P->W, H = P->H, D = P->D, Ds = P->Ds;
    int dx = OR_DX[r], dy = OR_DY[r];
    int P1 = P->p1;
    /* starting pixels: p - r lies outside the image */
    int nstart = 0;
    int* sx = (int*)malloc(sizeof(int) * (size_t)(W + H) * 2);
    int* sy = (int*)malloc(sizeof(int) * (size_t)(W + H) * 2);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int px = x - dx, py = y - dy;
            if (px < 0 || px >= W || py < 0 || py >= H) { sx[nstart] = x; sy[nstart] = y; ++nstart; }
        }
#pragma omp parallel
    {
        uint32_t* Lp = (uint32_t*)malloc(sizeof(uint32_t) * D);
        uint32_t* Lc = (uint32_t*)malloc(sizeof(uint32_t) * D);
#pragma omp for schedule(dynamic, 4)
        for (int i = 0; i < nstart; ++i) {
            int x = sx[i], y = sy[i];
            int step = 0;
            int g1 = 0, g2 = 0; /* g(p - r), g(p - 2r) */
            while (x >= 0 && x < W && y >= 0 && y < H) {
                size_t p = (size_t)y * W + x;
                const uint16_t* Sp = S + p * Ds;
                if (step == 0) {
                    for (int s = 0; s < D; ++s) Lc[s] = Sp[s];
                } else {
                    size_t q = (size_t)(y - dy) * W + (x - dx);
                    int di = 0;
                    if (P->variant == 1 && dI) di = dI[(size_t)r * W * H + p];
                    if (P->variant == 2 && step >= 2) di = g2 - g1;
                    if (di > P->dmax) di = P->dmax;
                    if (di < -P->dmax) di = -P->dmax;
                    int sh = (lo ? lo[p] - lo[q] : 0) + di;
                    int P2 = P->p2;
                    if (lut) {
                        int d = (int)img[p] - (int)img[q];
                        P2 = lut[d < 0 ? -d : d];
                    }
                    if (P2 < P1) P2 = P1;
                    sgm_step(Lp, D, sh, P1, P2, Sp, Lc);
                }
                for (int s = 0; s < D; ++s) acc[p * D + s] += Lc[s];
                if (Lout) memcpy(Lout + p * D, Lc, sizeof(uint32_t) * D);
                g2 = g1;
                g1 = (lo ? lo[p] : 0) + argmin_u32(Lc, D);
                uint32_t* tmp = Lp; Lp = Lc; Lc = tmp;
                x += dx;
                y += dy;
                ++step;
            }
        }
        free(Lp);
        free(Lc);
    }
    free(sx);
    free(sy);
}

/* Full aggregation: Sbar (uint16, H*W*Ds; slots >= D are written 0).
   Returns -2 if a sum does not fit 16 bits. */
OR_EXPORT int or_sgm_aggregate(const uint16_t* S, const int32_t* lo, const int8_t* dI,
                               const uint8_t* img, const uint16_t* lut, const or_sgm_params* P,
                               uint16_t* Sbar)
{
    size_t n = (size_t)P->W * P->H * P->D;
    uint32_t* acc = (uint32_t*)calloc(n, sizeof(uint32_t));
    for (int r = 0; r < P->paths; ++r) sgm_direction(S, lo, dI, img, lut, P, r, acc, NULL);
    int rc = 0;
    size_t np = (size_t)P->W * P->H;
    for (size_t p = 0; p < np; ++p)
        for (int s = 0; s < P->Ds; ++s) {
            uint32_t v = s < P->D ? acc[p * P->D + s] : 0;
            if (v > 65535u) rc = -2;
            Sbar[p * P->Ds + s] = (uint16_t)v;
        }
    free(acc);
    return rc;
}

/* L_r of a single direction (uint32, H*W*D) -- used by the tests */
OR_EXPORT void or_sgm_path(const uint16_t* S, const int32_t* lo, const int8_t* dI,
                           const uint8_t* img, const uint16_t* lut, const or_sgm_params* P, int r,
                           uint32_t* L)
{
    size_t n = (size_t)P->W * P->H * P->D;
    uint32_t* acc = (uint32_t*)calloc(n, sizeof(uint32_t));
    sgm_direction(S, lo, dI, img, lut, P, r, acc, L);
    free(acc);
}

/* ------------------------------------------------------------------------ */
/* Eq. sgm-wta, the depth of a plane (Sec. 2.3.2) and the depth refinement   */
/* (Sec. 2.3.4): winner-takes-all over the aggregated costs (lowest index on */
/* ties), then a parabola through the winner and its two neighbours, with    */
/* the samples placed at their plane distances delta (they are not equally  */
/* spaced).  Readings: no refinement at a window edge or when the parabola   */
/* is flat or opens downward; the vertex is clamped between the neighbours.  */
/* The vertex is the three-point parabolic step (as in Brent's method) with  */
/* xm = delta(g-1) > x0 = delta(g) > xp = delta(g+1).                        */
/* Depth d = -delta / (n^T K^-1 (x, y, 1)^T).                                */
/* ------------------------------------------------------------------------ */
OR_EXPORT double or_parabola_vertex(double xm, double cm, double x0, double c0, double xp, double cp)
{
    double a = (x0 - xm) * (c0 - cp);
    double b = (x0 - xp) * (c0 - cm);
    double den = a - b;
    if (!(den > 0.0)) return x0;
    double v = x0 - 0.5 * ((x0 - xm) * a - (x0 - xp) * b) / den;
    double lo = xm < xp ? xm : xp, hi = xm < xp ? xp : xm;
    if (v < lo) v = lo;
    if (v > hi) v = hi;
    return v;
}

OR_EXPORT void or_wta_refine(const uint16_t* Sbar, const int32_t* lo, int W, int H, int D, int Ds,
                             const double K[9], const double n[3], double rho0, double drho,
                             float* depth, int32_t* gwin)
{
    double fx = K[0], fy = K[4], cx = K[2], cy = K[5];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            const uint16_t* c = Sbar + p * Ds;
            int s = 0;
            for (int k = 1; k < D; ++k) if (c[k] < c[s]) s = k;
            int g = (lo ? lo[p] : 0) + s;
            double x0 = plane_delta(rho0, drho, g);
            double dl = x0;
            if (s > 0 && s < D - 1)
                dl = or_parabola_vertex(plane_delta(rho0, drho, g - 1), c[s - 1], x0, c[s],
                                        plane_delta(rho0, drho, g + 1), c[s + 1]);
            double ray = n[0] * (x - cx) / fx + n[1] * (y - cy) / fy + n[2];
            depth[p] = (float)(-dl / ray);
            if (gwin) gwin[p] = g;
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: 5x5 median filter on the refined depth map (clamp-to-edge).    */
/* ------------------------------------------------------------------------ */
static int cmp_float(const void* a, const void* b)
{
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

OR_EXPORT void or_median5(const float* in, int W, int H, float* out)
{
    float v[25];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int m = 0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i)
                    v[m++] = in[(size_t)clampi(y + j, 0, H - 1) * W + clampi(x + i, 0, W - 1)];
            qsort(v, 25, sizeof(float), cmp_float);
            out[(size_t)y * W + x] = v[12];
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4, Eq. normal and Eq. normal-smooth: back-project the depth map,   */
/* n_p = h_p x v_p from the horizontal and vertical neighbour differences,  */
/* then an appearance-weighted Gaussian smoothing                            */
/*   n_bar = n_p + sum_{q in W_p} n_q (2 pi s^2)^-1/2                        */
/*                   exp(-|q - p|^2 / (2 s^2) - |I(p) - I(q)| / beta)        */
/* and normalisation.  Readings: central differences (one-sided at the      */
/* border); the raw normal is turned to face the camera (n^T X(p) < 0); W_p */
/* is the (2r+1)^2 window including p, out-of-image q are skipped; sigma =   */
/* r (the paper fixes sigma to the window radius); a zero vector marks an   */
/* invalid normal (0, 0, 0).                                                 */
/* ------------------------------------------------------------------------ */
static void backproject(const float* depth, int W, int x, int y, double fx, double fy,
                        double cx, double cy, double* X)
{
    double d = depth[(size_t)y * W + x];
    X[0] = d * (x - cx) / fx;
    X[1] = d * (y - cy) / fy;
    X[2] = d;
}

OR_EXPORT void or_normals_raw(const float* depth, int W, int H, const double K[9], double* nrm)
{
    double fx = K[0], fy = K[4], cx = K[2], cy = K[5];
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double A[3], B[3], C[3], E[3], P[3], h[3], v[3], c[3];
            backproject(depth, W, clampi(x + 1, 0, W - 1), y, fx, fy, cx, cy, A);
            backproject(depth, W, clampi(x - 1, 0, W - 1), y, fx, fy, cx, cy, B);
            backproject(depth, W, x, clampi(y + 1, 0, H - 1), fx, fy, cx, cy, C);
            backproject(depth, W, x, clampi(y - 1, 0, H - 1), fx, fy, cx, cy, E);
            backproject(depth, W, x, y, fx, fy, cx, cy, P);
            for (int i = 0; i < 3; ++i) { h[i] = A[i] - B[i]; v[i] = C[i] - E[i]; }
            c[0] = h[1] * v[2] - h[2] * v[1];
            c[1] = h[2] * v[0] - h[0] * v[2];
            c[2] = h[0] * v[1] - h[1] * v[0];
            double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
            double* o = nrm + 3 * ((size_t)y * W + x);
            if (!(len > 0.0)) { o[0] = o[1] = o[2] = 0.0; continue; }
            double sgn = (c[0] * P[0] + c[1] * P[1] + c[2] * P[2]) > 0.0 ? -1.0 : 1.0;
            for (int i = 0; i < 3; ++i) o[i] = sgn * c[i] / len;
        }
}

/* Eq. normal-smooth on a given raw normal field nr [H][W][3]: the pixel's own
   normal plus the Gaussian- and appearance-weighted sum over the window of
   radius `radius` (p included, out-of-image q skipped), sigma = radius,
   weight (2 pi sigma^2)^-1/2 exp(-|q - p|^2 / (2 sigma^2) - |I_p - I_q| / beta);
   Eq. normal then normalises (a zero sum stays zero). */
OR_EXPORT void or_normals_smooth(const double* nr, const uint8_t* img, int W, int H, int radius, double beta,
                                 float* normal_out)
{
    double sigma = (double)radius;
    double norm = 1.0 / sqrt(2.0 * M_PI * sigma * sigma);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            double s[3] = {nr[3 * p], nr[3 * p + 1], nr[3 * p + 2]};
            for (int j = -radius; j <= radius; ++j)
                for (int i = -radius; i <= radius; ++i) {
                    int xx = x + i, yy = y + j;
                    if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                    size_t q = (size_t)yy * W + xx;
                    double dI = fabs((double)img[p] - (double)img[q]);
                    double wgt = norm * exp(-(double)(i * i + j * j) / (2.0 * sigma * sigma) - dI / beta);
                    for (int c = 0; c < 3; ++c) s[c] += nr[3 * q + c] * wgt;
                }
            double len = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
            for (int c = 0; c < 3; ++c) normal_out[3 * p + c] = len > 0.0 ? (float)(s[c] / len) : 0.0f;
        }
}

OR_EXPORT void or_normals(const float* depth, const uint8_t* img, int W, int H, const double K[9],
                          int radius, double beta, float* normal_out, float* raw_out)
{
    double* nr = (double*)malloc(sizeof(double) * 3 * (size_t)W * H);
    or_normals_raw(depth, W, H, K, nr);
    or_normals_smooth(nr, img, W, H, radius, beta, normal_out);
    if (raw_out)
        for (size_t i = 0; i < 3 * (size_t)W * H; ++i) raw_out[i] = (float)nr[i];
    free(nr);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.5, Eq. weight-normal: C = (<n_p,n_Pi><n_Pi,v> - cos rho) /         */
/* (1 - cos rho) when both angles are <= rho, else 0; v = (0,0,-1).         */
/* Reading: the result is clamped to [0, 1], the range the paper states.    */
/* ------------------------------------------------------------------------ */
OR_EXPORT void or_confidence(const float* normal, int W, int H, const double nPi[3], double rho_deg,
                             float* conf)
{
    double cr = cos(rho_deg * M_PI / 180.0);
    double b = -nPi[2];                       /* <n_Pi, v> */
    for (size_t p = 0; p < (size_t)W * H; ++p) {
        const float* np = normal + 3 * p;
        double a = np[0] * nPi[0] + np[1] * nPi[1] + np[2] * nPi[2];
        double c = 0.0;
        if (a >= cr && b >= cr) {
            c = (a * b - cr) / (1.0 - cr);
            if (c < 0.0) c = 0.0;
            if (c > 1.0) c = 1.0;
        }
        conf[p] = (float)c;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1, Eq. sampling_range and the dynamic cost volume (Sec. 2.2.1):    */
/* below the top level, pixel p samples a window of D planes around the      */
/* nearest-neighbour upscaled depth of the coarser level.  Reading: the     */
/* window is the D consecutive planes of the level list centred on the      */
/* plane nearest to that depth: c = (rho(d) - rho0) / drho,                 */
/* lo = clamp(floor(c + 1/2) - floor(D / 2), 0, G - D), with rho(d) the     */
/* inverse distance of the sweep plane through the back-projected point.    */
/* The decision is taken in FP32, every operation IEEE-rounded, in this      */
/* order: w = -(n0 a + n1 b + n2), a = (x - cx)/fx, b = (y - cy)/fy;         */
/* rho = 1 / (d w); c = (rho - rho0) / drho; floor(c + 0.5).                 */
/* ------------------------------------------------------------------------ */
static float ray_weight_f32(float n0, float n1, float n2, int x, int y, float fx, float fy,
                            float cx, float cy)
{
    volatile float a = ((float)x - cx) / fx;
    volatile float b = ((float)y - cy) / fy;
    volatile float m0 = n0 * a;
    volatile float m1 = n1 * b;
    volatile float s = m0 + m1;
    volatile float w = s + n2;
    return -w;
}

OR_EXPORT void or_window(const float* dc, int Wc, int Hc, int W, int H, const double K[9],
                         const double n[3], double rho0, double drho, int G, int D, int32_t* lo)
{
    float fx = (float)K[0], fy = (float)K[4], cx = (float)K[2], cy = (float)K[5];
    float n0 = (float)n[0], n1 = (float)n[1], n2 = (float)n[2];
    float r0 = (float)rho0, dr = (float)drho;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int xc = x / 2 < Wc - 1 ? x / 2 : Wc - 1, yc = y / 2 < Hc - 1 ? y / 2 : Hc - 1;
            float d = dc[(size_t)yc * Wc + xc];
            float w = ray_weight_f32(n0, n1, n2, x, y, fx, fy, cx, cy);
            volatile float t1 = d * w;
            volatile float rho = 1.0f / t1;
            volatile float t2 = rho - r0;
            volatile float c = t2 / dr;
            volatile float c5 = c + 0.5f;
            float fl = floorf(c5);
            int l;
            if (!(fl > -1.0e9f)) l = 0;             /* NaN or -inf */
            else if (fl > 1.0e9f) l = G - D;
            else l = (int)fl - D / 2;
            lo[(size_t)y * W + x] = clampi(l, 0, G - D);
        }
}

/* ------------------------------------------------------------------------ */
/* Eq. sgm-smooth-sn: the index jump di_sn caused by the tangent plane of    */
/* the prior normal n (from the coarser level) between p and its path        */
/* predecessor p - r.  The paper gives no formula; reading: with             */
/* P = d K^-1 (x, y, 1)^T, the predecessor ray meets the tangent plane       */
/* n^T X = n^T P at lambda K^-1 (p - r, 1)^T, and di is the change of the    */
/* sweep index 1/delta between the two points, delta = -m^T X for the sweep  */
/* normal m.  With s0 = n^T K^-1 (p,1), s1 = n^T K^-1 (r,0), u0 = m^T K^-1    */
/* (p,1), u1 = m^T K^-1 (r,0):                                              */
/*   di = round((s1 u0 - s0 u1) / (d s0 u0 (u0 - u1) drho)),                */
/* which for the fronto sweep m = (0,0,-1) (u0 = -1, u1 = 0) is             */
/* round(-s1 / (d s0 drho)) = round((1/lambda - 1/d) / drho), operation for  */
/* operation.  Rounded half away from zero and clamped to +-dmax; di = 0 for */
/* a zero normal or when the tangent plane or the sweep planes do not face   */
/* the two rays (s0, s0 - s1, u0 or u0 - u1 >= -1e-6).  Taken in FP32 with  */
/* every operation IEEE-rounded in the order written below.                  */
/* Output layout: int8 [8][H][W] in the path order of the aggregation.      */
/* ------------------------------------------------------------------------ */
OR_EXPORT void or_dsn(const float* dc, const float* nc, int Wc, int Hc, int W, int H,
                      const double K[9], const double m[3], double drho, int dmax, int8_t* dI)
{
    float fx = (float)K[0], fy = (float)K[4], cx = (float)K[2], cy = (float)K[5];
    float sw0 = (float)m[0], sw1 = (float)m[1], sw2 = (float)m[2];
    float dr = (float)drho;
    for (int r = 0; r < 8; ++r)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int xc = x / 2 < Wc - 1 ? x / 2 : Wc - 1, yc = y / 2 < Hc - 1 ? y / 2 : Hc - 1;
                size_t pc = (size_t)yc * Wc + xc;
                float d = dc[pc];
                float n0 = nc[3 * pc], n1 = nc[3 * pc + 1], n2 = nc[3 * pc + 2];
                int out = 0;
                volatile float a = ((float)x - cx) / fx;
                volatile float b = ((float)y - cy) / fy;
                volatile float m0 = n0 * a;
                volatile float m1 = n1 * b;
                volatile float s01 = m0 + m1;
                volatile float s0 = s01 + n2;                     /* n^T K^-1 (p,1) */
                volatile float gx = (float)OR_DX[r] / fx;
                volatile float gy = (float)OR_DY[r] / fy;
                volatile float q0 = n0 * gx;
                volatile float q1 = n1 * gy;
                volatile float s1 = q0 + q1;                      /* n^T K^-1 (r,0) */
                volatile float sp = s0 - s1;                      /* n^T K^-1 (p-r,1) */
                volatile float w0 = sw0 * a;
                volatile float w1 = sw1 * b;
                volatile float u01 = w0 + w1;
                volatile float u0 = u01 + sw2;                    /* m^T K^-1 (p,1) */
                volatile float v0 = sw0 * gx;
                volatile float v1 = sw1 * gy;
                volatile float u1 = v0 + v1;                      /* m^T K^-1 (r,0) */
                volatile float uq = u0 - u1;                      /* m^T K^-1 (p-r,1) */
                if ((n0 != 0.0f || n1 != 0.0f || n2 != 0.0f) && s0 < -1e-6f && sp < -1e-6f && u0 < -1e-6f &&
                    uq < -1e-6f && d > 0.0f) {
                    volatile float den0 = d * s0;
                    volatile float den1 = den0 * u0;
                    volatile float den2 = den1 * uq;
                    volatile float den = den2 * dr;
                    volatile float e0 = s1 * u0;
                    volatile float e1 = s0 * u1;
                    volatile float num = e0 - e1;
                    volatile float c = num / den;
                    float rc = c >= 0.0f ? floorf(c + 0.5f) : -floorf(-c + 0.5f);
                    if (rc > (float)dmax) rc = (float)dmax;
                    if (rc < (float)-dmax) rc = (float)-dmax;
                    out = (int)rc;
                }
                dI[(size_t)r * W * H + (size_t)y * W + x] = (int8_t)out;
            }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.2.2: plane selection.  Planes are n^T X + delta = 0 in the         */
/* reference frame (P_ref = K [I | 0]); the fronto sweep is n = (0,0,-1),    */
/* where delta is the depth.  A point at parameter s on the ray             */
/* X = s K^-1 (u,v,1)^T lies on the plane delta when s = -delta / (n^T r).    */
/* ------------------------------------------------------------------------ */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* the viewing ray K^-1 (u, v, 1)^T of the reference camera */
static void ref_ray(const double K[9], double u, double v, double r[3])
{
    double Ki[9];
    mat3_inv(K, Ki);
    for (int i = 0; i < 3; ++i) r[i] = Ki[3 * i] * u + Ki[3 * i + 1] * v + Ki[3 * i + 2];
}

/* pixel centres of the four image corners */
static void corner_px(int W, int H, int c, double* u, double* v)
{
    *u = (c & 1) ? (double)(W - 1) : 0.0;
    *v = (c & 2) ? (double)(H - 1) : 0.0;
}

/* Eq. of the bounding planes: the reference view frustum between the fronto */
/* near and far planes at depths d_min and d_max has four corners on each,   */
/* X = d K^-1 (u, v, 1)^T at the image corners.  delta_min is the smallest   */
/* |n^T X| over the near corners.  Reading: delta_max is the LARGEST |n^T X|  */
/* over the far corners -- the equation prints min for both, which for any   */
/* slanted n would stop the sweep short of the far corners; n^T X is linear  */
/* and the frustum is the convex hull of its 8 corners, so these two values  */
/* enclose it.  Returns -1 when a corner ray does not meet the planes        */
/* (n^T r >= 0: the sweep direction has no component along that ray).        */
OR_EXPORT int or_plane_bounds(const double K[9], int W, int H, const double n[3], double d_min, double d_max,
                              double out[2])
{
    double lo = INFINITY, hi = 0.0;
    for (int c = 0; c < 4; ++c) {
        double u, v, r[3], Xn[3], Xf[3];
        corner_px(W, H, c, &u, &v);
        ref_ray(K, u, v, r);
        if (!(dot3(n, r) < 0.0)) return -1;
        for (int i = 0; i < 3; ++i) {
            Xn[i] = d_min * r[i];
            Xf[i] = d_max * r[i];
        }
        lo = fmin(lo, fabs(dot3(n, Xn)));
        hi = fmax(hi, fabs(dot3(n, Xf)));
    }
    out[0] = lo;
    out[1] = hi;
    return 0;
}

/* x_k = K (R X + t) in homogeneous form */
static void project_h(const double K[9], const double R[9], const double t[3], const double X[3], double x[3])
{
    double Y[3];
    for (int i = 0; i < 3; ++i) Y[i] = R[3 * i] * X[0] + R[3 * i + 1] * X[1] + R[3 * i + 2] * X[2] + t[i];
    for (int i = 0; i < 3; ++i) x[i] = K[3 * i] * Y[0] + K[3 * i + 1] * Y[1] + K[3 * i + 2] * Y[2];
}

/* sine of the angle between two rays given by their directions (App. A) */
static double sin_between(const double a[3], const double b[3])
{
    double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    return sqrt(dot3(c, c)) / (sqrt(dot3(a, a)) * sqrt(dot3(b, b)));
}

/* Alg. 2: plane distances such that consecutive planes move the image of    */
/* the extreme point by at most one pixel in camera k.  Cameras: X_k =       */
/* R_k X + t_k (k < ncam).  Readings: (a) p_ref and camera k are the corner  */
/* and camera with the longest image segment between the projections of    */
/* P_min and P_max (the disparity range; the paper names the largest         */
/* disparity, typically a corner, and the most distant camera); (b) the     */
/* epipole enters only through the ray from C_k towards C_ref, taken from    */
/* its homogeneous image K t_k, so a reference centre behind camera k needs  */
/* no special case; (c) the walk takes whole steps p_i = p_max + i k for     */
/* i = 0 .. ceil(L) - 1 (L the segment length) and then ends ON p_min with   */
/* delta_min, so the last step is at most one pixel and both bounding planes */
/* are in the list.  The distance of each step follows from the cross-ratio: */
/* Q = delta (dmax - dmin) / (dmax (delta - dmin)) solved for delta.         */
/* Every camera centre must lie in front of Pi_min: n^T C_i + delta_min > 0. */
/* out[] gets the list far to near (delta_max first); returns the count, or  */
/* -1 (a camera centre behind Pi_min), -2 (a corner ray misses the planes),  */
/* -3 (no corner segment in any camera), -4 (more than maxn planes).         */
OR_EXPORT int or_cross_ratio_planes(const double K[9], int W, int H, int ncam, const double* R, const double* t,
                                    const double n[3], double delta_min, double delta_max, int maxn, double* out,
                                    int* chosen)
{
    for (int i = 0; i < ncam; ++i) {
        const double* Ri = R + 9 * i;
        const double* ti = t + 3 * i;
        double Ci[3];
        for (int j = 0; j < 3; ++j) Ci[j] = -(Ri[j] * ti[0] + Ri[3 + j] * ti[1] + Ri[6 + j] * ti[2]);
        if (!(dot3(n, Ci) + delta_min > 0.0)) return -1;
    }
    /* reading (a): camera k and p_ref */
    int k = -1;
    double best = 0.0, pu = 0.0, pv = 0.0;
    for (int i = 0; i < ncam; ++i)
        for (int c = 0; c < 4; ++c) {
            double u, v, r[3], Pn[3], Pf[3], xn[3], xf[3];
            corner_px(W, H, c, &u, &v);
            ref_ray(K, u, v, r);
            const double nr = dot3(n, r);
            if (!(nr < 0.0)) return -2;
            for (int j = 0; j < 3; ++j) {
                Pn[j] = r[j] * (-delta_min / nr);
                Pf[j] = r[j] * (-delta_max / nr);
            }
            project_h(K, R + 9 * i, t + 3 * i, Pn, xn);
            project_h(K, R + 9 * i, t + 3 * i, Pf, xf);
            if (!(xn[2] > 0.0 && xf[2] > 0.0)) continue;
            const double len = hypot(xn[0] / xn[2] - xf[0] / xf[2], xn[1] / xn[2] - xf[1] / xf[2]);
            if (len > best) {
                best = len;
                k = i;
                pu = u;
                pv = v;
            }
        }
    if (k < 0) return -3;
    if (chosen) *chosen = k;
    const double* Rk = R + 9 * k;
    const double* tk = t + 3 * k;
    /* step 1: the viewing ray through p_ref meets Pi_min and Pi_max */
    double V[3], Pmin[3], Pmax[3];
    ref_ray(K, pu, pv, V);
    const double nV = dot3(n, V);
    for (int j = 0; j < 3; ++j) {
        Pmin[j] = V[j] * (-delta_min / nV);
        Pmax[j] = V[j] * (-delta_max / nV);
    }
    /* step 2: images of C_ref, P_min and P_max in camera k */
    const double Cref[3] = {0.0, 0.0, 0.0};
    double eh[3], xmin[3], xmax[3];
    project_h(K, Rk, tk, Cref, eh);
    project_h(K, Rk, tk, Pmin, xmin);
    project_h(K, Rk, tk, Pmax, xmax);
    const double pmin[2] = {xmin[0] / xmin[2], xmin[1] / xmin[2]};
    const double pmax[2] = {xmax[0] / xmax[2], xmax[1] / xmax[2]};
    /* step 3: unit vector along the epipolar line, from p_max to p_min */
    const double L = hypot(pmin[0] - pmax[0], pmin[1] - pmax[1]);
    const double kx = (pmin[0] - pmax[0]) / L, ky = (pmin[1] - pmax[1]) / L;
    /* rays of camera k (directions in its own frame, K^-1 x) */
    double Kinv[9], Ve[3], Vmin[3], Vmax[3];
    mat3_inv(K, Kinv);
    for (int j = 0; j < 3; ++j) {
        Ve[j] = Kinv[3 * j] * eh[0] + Kinv[3 * j + 1] * eh[1] + Kinv[3 * j + 2] * eh[2];
        Vmin[j] = Kinv[3 * j] * pmin[0] + Kinv[3 * j + 1] * pmin[1] + Kinv[3 * j + 2];
        Vmax[j] = Kinv[3 * j] * pmax[0] + Kinv[3 * j + 1] * pmax[1] + Kinv[3 * j + 2];
    }
    const int steps = (int)ceil(L);
    if (steps + 1 > maxn) return -4;
    int m = 0;
    for (int i = 0; i < steps; ++i) {
        const double pi[2] = {pmax[0] + i * kx, pmax[1] + i * ky};
        double Vi[3];
        for (int j = 0; j < 3; ++j) Vi[j] = Kinv[3 * j] * pi[0] + Kinv[3 * j + 1] * pi[1] + Kinv[3 * j + 2];
        const double Q = sin_between(Ve, Vi) * sin_between(Vmin, Vmax) /
                         (sin_between(Ve, Vmax) * sin_between(Vmin, Vi));
        out[m++] = Q * delta_max * delta_min / (Q * delta_max - (delta_max - delta_min));
    }
    out[m++] = delta_min;
    return m;
}

/* ------------------------------------------------------------------------ */
/* Post-filters (Sec. 2.6).                                                  */
/* ------------------------------------------------------------------------ */

/* Alg. 3 (DoG mask), readings: the 7x7 Gaussian has sigma 1.4 (the usual     */
/* value for 7 taps), quantised per axis to integer weights summing to 256   */
/* (as the pyramid's, R1) with clamp-to-edge; DoG = I - I_smooth, marked     */
/* where |DoG| > 0.5 grey level; speckles are 4-connected components; the    */
/* 3x3 dilation takes the maximum over the in-image neighbours; the          */
/* estimates are invalidated where the final mask is 0 (the algorithm's last */
/* step names the mask value 1, at odds with its stated purpose of removing  */
/* weakly textured areas).                                                   */
OR_EXPORT void or_dog_weights(int32_t w[7])
{
    double g[7], s = 0.0;
    for (int i = 0; i < 7; ++i) {
        const double x = i - 3;
        g[i] = exp(-x * x / (2.0 * 1.4 * 1.4));
        s += g[i];
    }
    int tot = 0;
    for (int i = 0; i < 7; ++i) {
        w[i] = (int32_t)floor(256.0 * g[i] / s + 0.5);
        tot += w[i];
    }
    w[3] += 256 - tot;                   /* exact unit sum, the centre absorbs the rounding */
}

/* components (4-connected) of pixels equal to `val` smaller than minsize take
   the other value */
static void speckle(uint8_t* m, int W, int H, uint8_t val, int minsize);
OR_EXPORT void or_speckle(uint8_t* m, int W, int H, int val, int minsize) { speckle(m, W, H, (uint8_t)val, minsize); }

static void speckle(uint8_t* m, int W, int H, uint8_t val, int minsize)
{
    const size_t np = (size_t)W * H;
    int32_t* stack = (int32_t*)malloc(np * sizeof(int32_t));
    int32_t* comp = (int32_t*)malloc(np * sizeof(int32_t));
    uint8_t* seen = (uint8_t*)calloc(np, 1);
    for (size_t s0 = 0; s0 < np; ++s0) {
        if (m[s0] != val || seen[s0]) continue;
        int top = 0, n = 0;
        stack[top++] = (int32_t)s0;
        seen[s0] = 1;
        while (top > 0) {
            const int32_t p = stack[--top];
            comp[n++] = p;
            const int x = p % W, y = p / W;
            const int nx[4] = {x - 1, x + 1, x, x}, ny[4] = {y, y, y - 1, y + 1};
            for (int k = 0; k < 4; ++k) {
                if (nx[k] < 0 || nx[k] >= W || ny[k] < 0 || ny[k] >= H) continue;
                const int32_t q = ny[k] * W + nx[k];
                if (m[q] == val && !seen[q]) {
                    seen[q] = 1;
                    stack[top++] = q;
                }
            }
        }
        if (n < minsize)
            for (int i = 0; i < n; ++i) m[comp[i]] = (uint8_t)(1 - val);
    }
    free(stack);
    free(comp);
    free(seen);
}

OR_EXPORT void or_dog_mask(const uint8_t* img, int W, int H, uint8_t* mask)
{
    int32_t w[7];
    or_dog_weights(w);
    const size_t np = (size_t)W * H;
    int64_t* tmp = (int64_t*)malloc(np * sizeof(int64_t));
    for (int y = 0; y < H; ++y)            /* horizontal pass (x 256) */
        for (int x = 0; x < W; ++x) {
            int64_t a = 0;
            for (int i = -3; i <= 3; ++i) a += (int64_t)w[i + 3] * img[(size_t)y * W + clampi(x + i, 0, W - 1)];
            tmp[(size_t)y * W + x] = a;
        }
    for (int y = 0; y < H; ++y)            /* vertical pass (x 65536) and threshold */
        for (int x = 0; x < W; ++x) {
            int64_t a = 0;
            for (int j = -3; j <= 3; ++j) a += (int64_t)w[j + 3] * tmp[(size_t)clampi(y + j, 0, H - 1) * W + x];
            const int64_t dog = ((int64_t)img[(size_t)y * W + x] << 16) - a;
            mask[(size_t)y * W + x] = (dog > 32768 || dog < -32768) ? 1 : 0;
        }
    free(tmp);
    speckle(mask, W, H, 1, 7);             /* activation areas below 7 px */
    uint8_t* d = (uint8_t*)malloc(np);
    for (int y = 0; y < H; ++y)            /* 3x3 dilation */
        for (int x = 0; x < W; ++x) {
            uint8_t v = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) {
                    const int xx = x + i, yy = y + j;
                    if (xx >= 0 && xx < W && yy >= 0 && yy < H && mask[(size_t)yy * W + xx]) v = 1;
                }
            d[(size_t)y * W + x] = v;
        }
    memcpy(mask, d, np);
    free(d);
    speckle(mask, W, H, 0, 21);            /* deactivation areas below 21 px */
}

/* invalidates (sets to 0) the estimates where mask == 0 */
OR_EXPORT void or_apply_mask(const uint8_t* mask, int W, int H, float* depth, float* normal, float* conf)
{
    for (size_t p = 0; p < (size_t)W * H; ++p)
        if (!mask[p]) {
            depth[p] = 0.0f;
            normal[3 * p] = normal[3 * p + 1] = normal[3 * p + 2] = 0.0f;
            conf[p] = 0.0f;
        }
}

/* Alg. 4 (geometric consistency by mutual reprojection), readings: pixel p
   with depth d (z in the reference frame) is lifted to X = d K^-1 (x, y, 1),
   moved into view k (X_k = R_k X + t_k) and projected to p_k; the depth of
   map k is read at the pixel nearest to p_k (round half up), the point p_k is
   lifted with it and brought back: p~ = pi(R_k^T (X'_k - t_k)); a hit when
   |p - p~| < eta_r (pixels).  A point behind a camera, outside map k or on
   an invalid (<= 0) depth is a miss.  Fewer than eta_h hits invalidate p
   (depth, normal and confidence set to 0).  Every step in FP64 in the order
   written (the decision is an integer one).  K is shared by all maps. */
OR_EXPORT int or_geo_hits(const float* dref, int W, int H, const double K[9], int n,
                          const float* const* dk, const double* R, const double* t, double eta_r,
                          uint8_t* hits)
{
    const double fx = K[0], fy = K[4], cx = K[2], cy = K[5];
    if (K[1] != 0.0 || K[3] != 0.0 || K[6] != 0.0 || K[7] != 0.0 || K[8] != 1.0) return -1;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            int h = 0;
            const double d = dref[p];
            if (d > 0.0) {
                const double X0 = (x - cx) / fx * d, X1 = (y - cy) / fy * d, X2 = d;
                for (int k = 0; k < n; ++k) {
                    const double* Rk = R + 9 * k;
                    const double* tk = t + 3 * k;
                    const double Y0 = Rk[0] * X0 + Rk[1] * X1 + Rk[2] * X2 + tk[0];
                    const double Y1 = Rk[3] * X0 + Rk[4] * X1 + Rk[5] * X2 + tk[1];
                    const double Y2 = Rk[6] * X0 + Rk[7] * X1 + Rk[8] * X2 + tk[2];
                    if (!(Y2 > 0.0)) continue;
                    const double u = fx * Y0 / Y2 + cx, v = fy * Y1 / Y2 + cy;
                    const double ru = floor(u + 0.5), rv = floor(v + 0.5);
                    if (!(ru >= 0.0 && ru <= W - 1 && rv >= 0.0 && rv <= H - 1)) continue;
                    const double e = dk[k][(size_t)rv * W + (size_t)ru];
                    if (!(e > 0.0)) continue;
                    const double Z0 = (u - cx) / fx * e - tk[0], Z1 = (v - cy) / fy * e - tk[1], Z2 = e - tk[2];
                    const double B0 = Rk[0] * Z0 + Rk[3] * Z1 + Rk[6] * Z2;
                    const double B1 = Rk[1] * Z0 + Rk[4] * Z1 + Rk[7] * Z2;
                    const double B2 = Rk[2] * Z0 + Rk[5] * Z1 + Rk[8] * Z2;
                    if (!(B2 > 0.0)) continue;
                    const double du = fx * B0 / B2 + cx - x, dv = fy * B1 / B2 + cy - y;
                    if (sqrt(du * du + dv * dv) < eta_r) ++h;
                }
            }
            hits[p] = (uint8_t)h;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: the hierarchical loop.  From the coarsest level l = n-1 down to */
/* 0: plane-sweep cost volume (full plane list at the top level, per-pixel  */
/* windows below), SGM, WTA + refinement, 5x5 median, normals, confidence;  */
/* the depth and normal maps of level l, upscaled by nearest neighbour,     */
/* initialise level l-1.  Level l uses every 2^l-th plane of the finest     */
/* list (reading): G_l = floor((G0 - 1) / 2^l) + 1, drho_l = 2^l drho.      */
typedef struct {
    int32_t levels;
    int32_t D[8];          /* window size per level (the top level uses G_top) */
    int32_t paths;
    int32_t variant;
    int32_t p1, p2;        /* base penalties, multiplied by n_max here */
    int32_t adaptive_p2;
    double alpha, beta;
    int32_t median5;
    int32_t normal_radius;
    double normal_beta;
    double rho_deg;
    int32_t dmax;
    int32_t cost;          /* 0: census 9x7 (Hamming), 1: NCC 5x5 */
} or_config;

OR_EXPORT int or_estimate(const or_config* cfg, const uint8_t* ref, const uint8_t* const* nbrs,
                          int V, const int8_t* side, int W, int H, const double K[9],
                          const double* R, const double* t, const double n[3], double rho_far,
                          double drho, int G0, float* depth_out, float* normal_out, float* conf_out)
{
    int L = cfg->levels;
    if (L < 1 || L > 8) return -1;
    if ((G0 - 1) / (1 << (L - 1)) + 1 > 256) return -1;   /* 256-plane cap at the top (Sec. 3.2) */
    const uint8_t* imgs[8][17];          /* reference + up to 16 views per level */
    int Ws[8], Hs[8];
    uint8_t* owned[8 * 17];
    int nowned = 0;
    if (V < 1 || V > 16) return -1;
    imgs[0][0] = ref;
    for (int k = 0; k < V; ++k) imgs[0][k + 1] = nbrs[k];
    Ws[0] = W;
    Hs[0] = H;
    for (int l = 1; l < L; ++l) {
        Ws[l] = (Ws[l - 1] + 1) / 2;
        Hs[l] = (Hs[l - 1] + 1) / 2;
        for (int k = 0; k <= V; ++k) {
            uint8_t* o = (uint8_t*)malloc((size_t)Ws[l] * Hs[l]);
            or_pyramid_down(imgs[l - 1][k], Ws[l - 1], Hs[l - 1], o);
            imgs[l][k] = o;
            owned[nowned++] = o;
        }
    }
    int nL = 0, nR = 0;
    for (int k = 0; k < V; ++k) { if (side[k] < 0) ++nL; else ++nR; }
    int nmax = nL > nR ? nL : nR;
    int P1 = cfg->p1 * nmax;
    uint16_t lut[256];
    if (cfg->adaptive_p2) or_p2_table(P1, cfg->alpha, cfg->beta, lut);
    float* dprev = NULL;
    float* nprev = NULL;
    int rc = 0;
    for (int l = L - 1; l >= 0; --l) {
        int w = Ws[l], h = Hs[l];
        size_t np = (size_t)w * h;
        double s = (double)(1 << l);
        double Kl[9] = {K[0] / s, K[1], K[2] / s, K[3], K[4] / s, K[5] / s, 0.0, 0.0, 1.0};
        int Gl = (G0 - 1) / (1 << l) + 1;
        double drl = drho * s;
        int D = (l == L - 1) ? Gl : (cfg->D[l] < Gl ? cfg->D[l] : Gl);
        int32_t* lo = (int32_t*)calloc(np, sizeof(int32_t));
        int8_t* dI = NULL;
        if (l < L - 1) {
            or_window(dprev, Ws[l + 1], Hs[l + 1], w, h, Kl, n, rho_far, drl, Gl, D, lo);
            if (cfg->variant == 1) {
                dI = (int8_t*)malloc(8 * np);
                or_dsn(dprev, nprev, Ws[l + 1], Hs[l + 1], w, h, Kl, n, drl, cfg->dmax, dI);
            }
        }
        uint16_t* S = (uint16_t*)malloc(sizeof(uint16_t) * np * D);
        uint16_t* Sb = (uint16_t*)malloc(sizeof(uint16_t) * np * D);
        or_cost_volume(imgs[l][0], (const uint8_t* const*)&imgs[l][1], V, side, w, h, Kl, R, t, n,
                       rho_far, drl, Gl, lo, D, D, cfg->cost, S);
        or_sgm_params P = {w, h, D, D, Gl, cfg->paths, cfg->variant, P1, cfg->p2 * nmax, cfg->dmax};
        if (or_sgm_aggregate(S, lo, dI, imgs[l][0], cfg->adaptive_p2 ? lut : NULL, &P, Sb) != 0) rc = -2;
        float* draw = (float*)malloc(sizeof(float) * np);
        float* dmed = (float*)malloc(sizeof(float) * np);
        float* nrm = (float*)malloc(sizeof(float) * 3 * np);
        or_wta_refine(Sb, lo, w, h, D, D, Kl, n, rho_far, drl, draw, NULL);
        if (cfg->median5) or_median5(draw, w, h, dmed);
        else memcpy(dmed, draw, sizeof(float) * np);
        or_normals(dmed, imgs[l][0], w, h, Kl, cfg->normal_radius, cfg->normal_beta, nrm, NULL);
        if (l == 0) {
            memcpy(depth_out, dmed, sizeof(float) * np);
            memcpy(normal_out, nrm, sizeof(float) * 3 * np);
            or_confidence(nrm, w, h, n, cfg->rho_deg, conf_out);
        }
        free(dprev);
        free(nprev);
        dprev = dmed;
        nprev = nrm;
        free(draw);
        free(lo);
        free(dI);
        free(S);
        free(Sb);
    }
    free(dprev);
    free(nprev);
    for (int i = 0; i < nowned; ++i) free(owned[i]);
    return rc;
}
