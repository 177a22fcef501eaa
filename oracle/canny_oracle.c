/*
 * canny_oracle.c -- plain, single-threaded CPU Canny edge detector.
 *
 * TEST INFRASTRUCTURE: the checker for the CUDA library, never on its path.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline legs load
 * it. Built with -ffp-contract=off so that the float32 variant rounds every
 * product and sum separately, in the order written here.
 *
 * Paper: H. Mogale, "High Performance Canny Edge Detector using Parallel
 * Patterns for Scalability on Modern Multicore Processors", Sec. 2.2.1
 * (Algorithm 1 and Steps 1-4). Each stage below is the plain definition,
 * computed over the whole image into full-size arrays; nothing is fused,
 * blocked or reordered.
 *
 * All functions are pinned by tests (closed forms, scipy/numpy routines,
 * brute force, invariants); see the header.
 */
#include "canny_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ======================================================================== */
/* Integer path                                                             */
/* ======================================================================== */

/*
 * Step 1, "Filter out any noise" (Sec. 2.2.1; gaussianfilter in Algorithm 1).
 * The paper gives no kernel. Integer reading: the 5x5 binomial kernel
 * b_i * b_j with b = (1,4,6,4,1) (sum 256), applied directly as a 25-tap 2-D
 * sum, rounded half up by (acc + 128) >> 8. Pixels outside the image take the
 * value of the nearest edge pixel (replicate border), so a constant image
 * stays constant.
 */
void oracle_gauss5_u8(const uint8_t *img, int w, int h, int pitch, uint8_t *S)
{
    static const int b[5] = {1, 4, 6, 4, 1};
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int acc = 0;
            for (int i = -2; i <= 2; ++i) {
                int yy = clampi(y + i, 0, h - 1);
                for (int j = -2; j <= 2; ++j) {
                    int xx = clampi(x + j, 0, w - 1);
                    acc += b[i + 2] * b[j + 2] * (int)img[(int64_t)yy * pitch + xx];
                }
            }
            S[(int64_t)y * w + x] = (uint8_t)((acc + 128) >> 8);
        }
    }
}

/*
 * Step 2, "Obtain Gradient intensity" (Sec. 2.2.1): the Sobel pair (Gx, Gy).
 * x grows to the right and y downwards. The smoothed image S is read with the
 * same replicate border as Step 1 (S at the nearest in-image position).
 *   Gx = [S(x+1,y-1) + 2 S(x+1,y) + S(x+1,y+1)] - [same three at x-1]
 *   Gy = [S(x-1,y+1) + 2 S(x,y+1) + S(x+1,y+1)] - [same three at y-1]
 * Both lie in [-1020, 1020].
 */
void oracle_sobel_u8(const uint8_t *S, int w, int h, int16_t *gx, int16_t *gy)
{
    for (int y = 0; y < h; ++y) {
        int ym = clampi(y - 1, 0, h - 1), yp = clampi(y + 1, 0, h - 1);
        for (int x = 0; x < w; ++x) {
            int xm = clampi(x - 1, 0, w - 1), xp = clampi(x + 1, 0, w - 1);
#define SV(xx, yy) ((int)S[(int64_t)(yy) * w + (xx)])
            int right = SV(xp, ym) + 2 * SV(xp, y) + SV(xp, yp);
            int left = SV(xm, ym) + 2 * SV(xm, y) + SV(xm, yp);
            int down = SV(xm, yp) + 2 * SV(x, yp) + SV(xp, yp);
            int up = SV(xm, ym) + 2 * SV(x, ym) + SV(xp, ym);
#undef SV
            gx[(int64_t)y * w + x] = (int16_t)(right - left);
            gy[(int64_t)y * w + x] = (int16_t)(down - up);
        }
    }
}

/*
 * Step 2, gradient strength ("p <- G(x,y)" in Algorithm 1). Integer reading:
 * the squared L2 norm Gx^2 + Gy^2 (at most 2,080,800), so thresholds are
 * compared squared and no square root is taken.
 */
void oracle_mag2_i32(const int16_t *gx, const int16_t *gy, int64_t n, int32_t *m2)
{
    for (int64_t i = 0; i < n; ++i)
        m2[i] = (int32_t)gx[i] * gx[i] + (int32_t)gy[i] * gy[i];
}

/*
 * Step 2, gradient direction ("theta <- arctan(...)" in Algorithm 1), read as
 * the usual 4-sector quantisation of atan2(Gy, Gx) without computing an
 * arctangent. The sector boundary tan(22.5 deg) = sqrt(2) - 1 is held in Q15
 * fixed point: T = round((sqrt(2) - 1) * 2^15).
 */
int oracle_sector_tan_q15(void)
{
    return (int)lround((sqrt(2.0) - 1.0) * 32768.0);
}

/*
 *   H (compare left/right)     if |Gy| * 2^15 < |Gx| * T
 *   V (compare up/down)        if |Gx| * 2^15 < |Gy| * T
 *   D (compare (x-1,y-1), (x+1,y+1)) otherwise, when Gx and Gy have the same
 *                                    strict sign
 *   A (compare (x+1,y-1), (x-1,y+1)) otherwise.
 * The V test is the H test with the axes swapped, so a 90-degree rotation of
 * the gradient maps H<->V and D<->A exactly.
 */
int oracle_sector_i(int gx, int gy)
{
    const int64_t T = oracle_sector_tan_q15();
    int64_t ax = gx < 0 ? -(int64_t)gx : gx;
    int64_t ay = gy < 0 ? -(int64_t)gy : gy;
    if (ay * 32768 < ax * T) return ORACLE_SECTOR_H;
    if (ax * 32768 < ay * T) return ORACLE_SECTOR_V;
    if ((gx > 0 && gy > 0) || (gx < 0 && gy < 0)) return ORACLE_SECTOR_D;
    return ORACLE_SECTOR_A;
}

void oracle_sector_map_i(const int32_t *gx, const int32_t *gy, int64_t n, uint8_t *sec)
{
    for (int64_t i = 0; i < n; ++i) sec[i] = (uint8_t)oracle_sector_i(gx[i], gy[i]);
}

/* neighbour offsets (dx, dy) on the negative and positive side of each sector */
static const int nms_neg[4][2] = {{-1, 0}, {0, -1}, {-1, -1}, {-1, 1}};
static const int nms_pos[4][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}};

/*
 * Step 3, non-maximum suppression (Sec. 2.2.1), and the double threshold of
 * Step 4. A pixel survives if its strength beats the neighbour on the negative
 * side of its sector strictly and is at least the one on the positive side
 * (the negative side is the left, upper, upper-left (D) or lower-left (A)
 * pixel); a plateau thus keeps exactly its first pixel along the positive
 * direction. Neighbours outside the image count as strength 0.
 * Step 4 thresholds, strict: class STRONG if M2 > hi2, WEAK if lo2 < M2 <= hi2,
 * NONE otherwise or if suppressed.
 */
void oracle_nms_classify_u8(const int16_t *gx, const int16_t *gy, const int32_t *m2,
                            int w, int h, int64_t lo2, int64_t hi2, uint8_t *cls)
{
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int64_t i = (int64_t)y * w + x;
            int s = oracle_sector_i(gx[i], gy[i]);
            int64_t m = m2[i];
            int xn = x + nms_neg[s][0], yn = y + nms_neg[s][1];
            int xp = x + nms_pos[s][0], yp = y + nms_pos[s][1];
            int64_t mn = (xn >= 0 && xn < w && yn >= 0 && yn < h) ? m2[(int64_t)yn * w + xn] : 0;
            int64_t mp = (xp >= 0 && xp < w && yp >= 0 && yp < h) ? m2[(int64_t)yp * w + xp] : 0;
            int keep = (m > mn) && (m >= mp);
            uint8_t c = ORACLE_NONE;
            if (keep && m > hi2) c = ORACLE_STRONG;
            else if (keep && m > lo2) c = ORACLE_WEAK;
            cls[i] = c;
        }
    }
}

/*
 * Step 4, hysteresis (Sec. 2.2.1): a pixel above the upper threshold is an
 * edge; one between the thresholds is an edge only if it is connected to one
 * above the upper threshold. Connectivity is read as 8-connectivity through
 * WEAK/STRONG pixels. FIFO breadth-first search from every STRONG pixel.
 * Output is 255 for an edge, 0 otherwise; bytes past w in each pitched row
 * are left untouched.
 */
void oracle_hysteresis(const uint8_t *cls, int w, int h, uint8_t *out, int out_pitch)
{
    int64_t n = (int64_t)w * h;
    uint8_t *edge = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < n; ++i)
        if (cls[i] == ORACLE_STRONG) { edge[i] = 1; queue[tail++] = i; }
    while (head < tail) {
        int64_t i = queue[head++];
        int y = (int)(i / w), x = (int)(i % w);
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = x + dx, yy = y + dy;
                if ((dx == 0 && dy == 0) || xx < 0 || xx >= w || yy < 0 || yy >= h) continue;
                int64_t j = (int64_t)yy * w + xx;
                if (!edge[j] && cls[j] != ORACLE_NONE) { edge[j] = 1; queue[tail++] = j; }
            }
    }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x)
            out[(int64_t)y * out_pitch + x] = edge[(int64_t)y * w + x] ? 255 : 0;
    free(queue);
    free(edge);
}

/* Steps 1-3 and the thresholds of Step 4: the class map before hysteresis. */
void oracle_classify_u8(const uint8_t *img, int w, int h, int pitch, int low, int high,
                        uint8_t *cls)
{
    int64_t n = (int64_t)w * h;
    if (n <= 0) return;
    uint8_t *S = (uint8_t *)malloc((size_t)n);
    int16_t *gx = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *gy = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int32_t *m2 = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    oracle_gauss5_u8(img, w, h, pitch, S);
    oracle_sobel_u8(S, w, h, gx, gy);
    oracle_mag2_i32(gx, gy, n, m2);
    oracle_nms_classify_u8(gx, gy, m2, w, h, (int64_t)low * low, (int64_t)high * high, cls);
    free(m2);
    free(gy);
    free(gx);
    free(S);
}

/* The whole integer pipeline, Steps 1-4: uint8 image in, 0/255 edge map out. */
void oracle_canny_u8(const uint8_t *img, int w, int h, int in_pitch, int low, int high,
                     uint8_t *out, int out_pitch)
{
    int64_t n = (int64_t)w * h;
    if (n <= 0) return;
    uint8_t *cls = (uint8_t *)malloc((size_t)n);
    oracle_classify_u8(img, w, h, in_pitch, low, high, cls);
    oracle_hysteresis(cls, w, h, out, out_pitch);
    free(cls);
}

/* ======================================================================== */
/* Float32 variant                                                          */
/* ======================================================================== */

/*
 * Step 1 with a sigma-parametrised Gaussian: taps g_k = exp(-k^2 / (2 sigma^2))
 * for k = -r..r, r = ksize / 2, normalised by their sum in double precision,
 * then rounded to float.
 */
void oracle_gauss_taps_f32(float sigma, int ksize, float *taps)
{
    int r = ksize / 2;
    double s = (double)sigma, g[64], sum = 0.0;
    for (int k = -r; k <= r; ++k) {
        g[k + r] = exp(-(double)(k * k) / (2.0 * s * s));
        sum += g[k + r];
    }
    for (int k = 0; k < ksize; ++k) taps[k] = (float)(g[k] / sum);
}

/*
 * Step 1, float32: separable, horizontal pass then vertical pass, replicate
 * border, each pass accumulating tap 0 first and every later product added
 * in float (one rounding per product and per sum). The input is float(u8),
 * not rescaled.
 */
void oracle_gauss_f32(const uint8_t *img, int w, int h, int pitch, float sigma, int ksize,
                      float *S)
{
    int r = ksize / 2;
    float taps[64];
    oracle_gauss_taps_f32(sigma, ksize, taps);
    float *tmp = (float *)malloc((size_t)w * h * sizeof(float));
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            float acc = taps[0] * (float)img[(int64_t)y * pitch + clampi(x - r, 0, w - 1)];
            for (int k = 1; k < ksize; ++k)
                acc = acc + taps[k] * (float)img[(int64_t)y * pitch + clampi(x - r + k, 0, w - 1)];
            tmp[(int64_t)y * w + x] = acc;
        }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            float acc = taps[0] * tmp[(int64_t)clampi(y - r, 0, h - 1) * w + x];
            for (int k = 1; k < ksize; ++k)
                acc = acc + taps[k] * tmp[(int64_t)clampi(y - r + k, 0, h - 1) * w + x];
            S[(int64_t)y * w + x] = acc;
        }
    free(tmp);
}

/*
 * Step 2, float32 Sobel with the same taps, border and axes as the integer
 * path. Order: the three taps of a column (or row) are summed top to bottom
 * (left to right), then the negative side is subtracted.
 */
void oracle_sobel_f32(const float *S, int w, int h, float *gx, float *gy)
{
    for (int y = 0; y < h; ++y) {
        int ym = clampi(y - 1, 0, h - 1), yp = clampi(y + 1, 0, h - 1);
        for (int x = 0; x < w; ++x) {
            int xm = clampi(x - 1, 0, w - 1), xp = clampi(x + 1, 0, w - 1);
#define SF(xx, yy) (S[(int64_t)(yy) * w + (xx)])
            float right = SF(xp, ym) + 2.0f * SF(xp, y);
            right = right + SF(xp, yp);
            float left = SF(xm, ym) + 2.0f * SF(xm, y);
            left = left + SF(xm, yp);
            float down = SF(xm, yp) + 2.0f * SF(x, yp);
            down = down + SF(xp, yp);
            float up = SF(xm, ym) + 2.0f * SF(x, ym);
            up = up + SF(xp, ym);
#undef SF
            gx[(int64_t)y * w + x] = right - left;
            gy[(int64_t)y * w + x] = down - up;
        }
    }
}

/* Step 2, float32 strength: M = sqrt(Gx*Gx + Gy*Gy), each operation rounded. */
void oracle_magnitude_f32(const float *gx, const float *gy, int64_t n, float *M)
{
    for (int64_t i = 0; i < n; ++i) {
        float xx = gx[i] * gx[i];
        float yy = gy[i] * gy[i];
        M[i] = sqrtf(xx + yy);
    }
}

/* The image's largest strength, over all pixels before suppression. */
float oracle_max_f32(const float *M, int64_t n)
{
    float m = 0.0f;
    for (int64_t i = 0; i < n; ++i)
        if (M[i] > m) m = M[i];
    return m;
}

/*
 * Step 2 direction, float32: the integer sector rule with tan(22.5 deg) taken
 * as the float 0.41421356f: H if |Gy| < |Gx| * t, V if |Gx| < |Gy| * t,
 * otherwise D (same strict sign) or A.
 */
int oracle_sector_f(float gx, float gy)
{
    const float t = 0.41421356f;
    float ax = fabsf(gx), ay = fabsf(gy);
    if (ay < ax * t) return ORACLE_SECTOR_H;
    if (ax < ay * t) return ORACLE_SECTOR_V;
    if ((gx > 0.0f && gy > 0.0f) || (gx < 0.0f && gy < 0.0f)) return ORACLE_SECTOR_D;
    return ORACLE_SECTOR_A;
}

/* Step 3 and the Step 4 thresholds, float32, same rules as the integer path. */
void oracle_nms_classify_f32(const float *gx, const float *gy, const float *M, int w, int h,
                             float lo_t, float hi_t, uint8_t *cls)
{
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            int64_t i = (int64_t)y * w + x;
            int s = oracle_sector_f(gx[i], gy[i]);
            float m = M[i];
            int xn = x + nms_neg[s][0], yn = y + nms_neg[s][1];
            int xp = x + nms_pos[s][0], yp = y + nms_pos[s][1];
            float mn = (xn >= 0 && xn < w && yn >= 0 && yn < h) ? M[(int64_t)yn * w + xn] : 0.0f;
            float mp = (xp >= 0 && xp < w && yp >= 0 && yp < h) ? M[(int64_t)yp * w + xp] : 0.0f;
            int keep = (m > mn) && (m >= mp);
            uint8_t c = ORACLE_NONE;
            if (keep && m > hi_t) c = ORACLE_STRONG;
            else if (keep && m > lo_t) c = ORACLE_WEAK;
            cls[i] = c;
        }
    }
}

/*
 * The whole float32 pipeline. Thresholds are fractions of the image's largest
 * strength Mmax: lo_t = lo_frac * Mmax, hi_t = hi_frac * Mmax (float products).
 * A flat image (Mmax = 0) has no edges. Optionally returns M and the class map.
 */
void oracle_canny_f32(const uint8_t *img, int w, int h, int in_pitch, float sigma, int ksize,
                      float lo_frac, float hi_frac, uint8_t *out, int out_pitch,
                      float *M_out, uint8_t *cls_out)
{
    int64_t n = (int64_t)w * h;
    if (n <= 0) return;
    float *S = (float *)malloc((size_t)n * sizeof(float));
    float *gx = (float *)malloc((size_t)n * sizeof(float));
    float *gy = (float *)malloc((size_t)n * sizeof(float));
    float *M = M_out ? M_out : (float *)malloc((size_t)n * sizeof(float));
    uint8_t *cls = cls_out ? cls_out : (uint8_t *)malloc((size_t)n);
    oracle_gauss_f32(img, w, h, in_pitch, sigma, ksize, S);
    oracle_sobel_f32(S, w, h, gx, gy);
    oracle_magnitude_f32(gx, gy, n, M);
    float mmax = oracle_max_f32(M, n);
    float lo_t = lo_frac * mmax, hi_t = hi_frac * mmax;
    oracle_nms_classify_f32(gx, gy, M, w, h, lo_t, hi_t, cls);
    oracle_hysteresis(cls, w, h, out, out_pitch);
    if (!cls_out) free(cls);
    if (!M_out) free(M);
    free(gy);
    free(gx);
    free(S);
}
