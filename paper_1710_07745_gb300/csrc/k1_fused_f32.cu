// k1_fused_f32.cu -- the float32 variant of Steps 1-4 (paper Sec. 2.2.1) without a
// stored strength image. The thresholds are fractions of the image's largest
// strength, a grid-wide dependency, so the stencil runs twice over the input:
//
//   pass 1 (k1f_max_kernel): Gaussian -> Sobel -> squared strength s = gx^2 + gy^2
//     for every pixel, reduced to the image maximum smax (one atomicMax per CTA);
//   pass 2 (k1f_edges_kernel): the same stencil again, then on the few pixels
//     that can pass the low threshold: strength M = sqrt(s), direction sector,
//     suppression, double threshold; then the tile flood fill of the hysteresis
//     on 32 x 32 tiles and the 0/255 edge bytes, tile border masks and pending
//     bitmaps for the global passes.
//
// Each pass reads the input byte once; pass 2 writes the edge byte once. The
// largest strength is Mmax = sqrt(smax) exactly: a correctly rounded square
// root is monotonic, so the largest root is the root of the largest s.
//
// Arithmetic follows the float32 definition operation by operation (no
// contraction except where a product by 2 is exact): horizontal pass then
// vertical pass, taps accumulated from the first, replicate border; Sobel
// columns summed top to bottom; s = (gx*gx) + (gy*gy); M = sqrt_rn(s).
//
// A CTA of 256 threads covers a block of 64 rows x 128 columns (2 x 4 tiles)
// and stages it in shared memory: input (as float, with a halo of R + 2 rows
// and R + 2 columns rounded up to 16, R = ksize / 2; 16-byte vector loads
// where the block lies inside the image), the horizontal pass, the smoothed
// image S, the squared strengths (with a 1-pixel ring for the suppression).
// Buffers alias once they are dead, so a 7-tap kernel needs 86 KB and two CTAs
// fit on an SM. Work is done on pixel pairs that share their shared-memory
// loads (the horizontal pass pairs two rows, the vertical pass and Sobel pair
// two columns); the arithmetic itself is scalar and correctly rounded per
// operation (__fmul_rn / __fadd_rn, and __fmaf_rn only where the product by 2
// is exact).
#include "hyst_tile.cuh"

namespace canny {

namespace {

constexpr int FB_W = 128, FB_H = 64;            // output block
constexpr int FB_THREADS = 256;
constexpr int FB_WARPS = FB_THREADS / 32;
constexpr int FB_TX = FB_W / HT, FB_TY = FB_H / HT;
static_assert(FB_TX * FB_TY == FB_WARPS, "one warp per tile in the flood stage");

struct Geometry {
    int R, padx, pady;         // Gaussian radius; input halo (columns rounded up to 4)
    int IY, IX;                // staged input rows / columns
    int SX, SY;                // smoothed image: columns x0-2 .. x0+FB_W+1, rows y0-2 .. y0+FB_H+1
    int MX, MY;                // squared strength with its ring, rows y0-1 .. y0+FB_H; column j is
                               // x0-2+j like S (the ring uses j = 1 .. FB_W+2), MX the row stride
    int region0, region1;      // floats: input then S; horizontal pass then s
};

__host__ __device__ inline Geometry geometry(int ksize)
{
    Geometry g;
    g.R = ksize / 2;
    g.pady = g.R + 2;
    g.padx = (g.R + 2 + 15) / 16 * 16;      // 16-byte aligned input rows
    g.IY = FB_H + 2 * g.pady;
    g.IX = FB_W + 2 * g.padx;
    g.SX = FB_W + 4;
    g.SY = FB_H + 4;
    g.MX = FB_W + 4;
    g.MY = FB_H + 2;
    const int a = g.IY * g.IX, b = g.SY * g.SX, c = g.IY * g.SX, d = g.MY * g.MX;
    g.region0 = a > b ? a : b;
    g.region1 = c > d ? c : d;
    return g;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// One Gaussian tap sum on a pair of independent sums:
// taps[0]*v(0) + taps[1]*v(1) + ..., each product and each sum rounded. The
// pair shares its loads; the arithmetic is scalar __fmul_rn / __fadd_rn per
// lane, which are never merged into a fused multiply-add (a paired multiply
// followed by a paired add was observed to round once, like an FMA).
// KS = 0: run-time ksize (taps read by index).
template <int KS, typename Load>
__device__ __forceinline__ float2 tap_sum2(const FloatParams &fp, Load v)
{
    float2 x = v(0);
    float2 acc = f2(fmul(fp.taps[0], x.x), fmul(fp.taps[0], x.y));
    if constexpr (KS > 0) {
#pragma unroll
        for (int k = 1; k < KS; ++k) {
            x = v(k);
            acc = f2(fadd(acc.x, fmul(fp.taps[k], x.x)), fadd(acc.y, fmul(fp.taps[k], x.y)));
        }
    } else {
        for (int k = 1; k < fp.ksize; ++k) {
            x = v(k);
            acc = f2(fadd(acc.x, fmul(fp.taps[k], x.x)), fadd(acc.y, fmul(fp.taps[k], x.y)));
        }
    }
    return acc;
}

// Sobel at the S entry (r, c) of a row-major S block with row stride sx, in the
// definition's order; a + 2*b is formed as fma(2, b, a), which is the same
// single rounding since 2*b is exact.
__device__ __forceinline__ void sobel_at(const float *S, int sx, int r, int c, float &gx, float &gy)
{
    const float *u = S + (r - 1) * sx + c, *m = S + r * sx + c, *d = S + (r + 1) * sx + c;
    float right = __fmaf_rn(2.f, m[1], u[1]);
    right = fadd(right, d[1]);
    float left = __fmaf_rn(2.f, m[-1], u[-1]);
    left = fadd(left, d[-1]);
    float down = __fmaf_rn(2.f, d[0], d[-1]);
    down = fadd(down, d[1]);
    float up = __fmaf_rn(2.f, u[0], u[-1]);
    up = fadd(up, u[1]);
    gx = fadd(right, -left);
    gy = fadd(down, -up);
}

__device__ __forceinline__ float strength2(float gx, float gy) { return fadd(fmul(gx, gx), fmul(gy, gy)); }

// Squared strengths of the pixel pair at S entries (r, c), (r, c + 1), c even:
// the operations of sobel_at + strength2 on each pixel, sharing the loads.
__device__ __forceinline__ float2 strength2_pair(const float *S, int sx, int r, int c)
{
    const float *u = S + (r - 1) * sx + c - 2, *m = S + r * sx + c - 2, *d = S + (r + 1) * sx + c - 2;
    // columns c-2 .. c+3 of rows r-1, r, r+1 as aligned pairs
    const float2 u0 = *reinterpret_cast<const float2 *>(u), u1 = *reinterpret_cast<const float2 *>(u + 2),
                 u2 = *reinterpret_cast<const float2 *>(u + 4);
    const float2 m0 = *reinterpret_cast<const float2 *>(m), m1 = *reinterpret_cast<const float2 *>(m + 2),
                 m2 = *reinterpret_cast<const float2 *>(m + 4);
    const float2 d0 = *reinterpret_cast<const float2 *>(d), d1 = *reinterpret_cast<const float2 *>(d + 2),
                 d2 = *reinterpret_cast<const float2 *>(d + 4);
    const float U[5] = {u0.y, u1.x, u1.y, u2.x, 0.f}, M[5] = {m0.y, m1.x, m1.y, m2.x, 0.f},
                D[5] = {d0.y, d1.x, d1.y, d2.x, 0.f};    // columns c-1 .. c+2
    float out[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {                      // pixel at column c + i: index 1 + i
        const float right = fadd(__fmaf_rn(2.f, M[2 + i], U[2 + i]), D[2 + i]);
        const float left = fadd(__fmaf_rn(2.f, M[i], U[i]), D[i]);
        const float down = fadd(__fmaf_rn(2.f, D[1 + i], D[i]), D[2 + i]);
        const float up = fadd(__fmaf_rn(2.f, U[1 + i], U[i]), U[2 + i]);
        out[i] = strength2(fadd(right, -left), fadd(down, -up));
    }
    return f2(out[0], out[1]);
}

// float(byte k of w), exactly: 2^23 + byte from a byte permute, minus 2^23.
__device__ __forceinline__ float byte_f(uint32_t w, int k)
{
    return __fadd_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7640u | (uint32_t)k)), -8388608.f);
}

// Horizontal pass of one row for NOUT consecutive outputs H[c0 .. c0+NOUT) at
// image columns x0 - 2 + c0 + q, straight from global memory: the 48 bytes from
// the 16-byte aligned column x0 + c0 - 16 hold every input these outputs read
// (for a radius up to 14). No clamping: the caller checks the block is inside.
template <int KS, int NOUT>
__device__ __forceinline__ void hrow_regs(const uint8_t *row, int x0, int c0, const FloatParams &fp, float *dst)
{
    constexpr int R = KS / 2;
    const uint4 *src = reinterpret_cast<const uint4 *>(row + x0 + c0 - 16);
    const uint4 a = __ldg(src), b = __ldg(src + 1), c = __ldg(src + 2);
    const uint32_t wd[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    // window index of image column x0 - 2 + c0 + q - R + k is 14 + q - R + k
    constexpr int LO = 14 - R, N = NOUT + 2 * R;
    float v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = byte_f(wd[(LO + i) >> 2], (LO + i) & 3);
    float out[NOUT];
#pragma unroll
    for (int q = 0; q < NOUT; ++q) {
        float acc = fmul(fp.taps[0], v[q]);
#pragma unroll
        for (int k = 1; k < KS; ++k) acc = fadd(acc, fmul(fp.taps[k], v[q + k]));
        out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < NOUT; q += 4)
        *reinterpret_cast<float4 *>(dst + q) = make_float4(out[q], out[q + 1], out[q + 2], out[q + 3]);
}

// Step 1's horizontal pass through a staged copy of the input (blocks at the
// image's left or right edge, or inputs without 16-byte alignment): the input
// block is staged as floats with clamped columns, then H is computed at the
// clamped columns, rows paired.
template <int KS>
__device__ __forceinline__ void staged_hpass(const uint8_t *__restrict__ in, int in_pitch, int w, int h,
                                             const FloatParams &fp, const Geometry &g, int x0, int y0,
                                             float *I_s, float *H_s, bool aligned)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ox = x0 - g.padx, oy = y0 - g.pady;
    const bool vec = ox >= 0 && ox + g.IX <= w && aligned;
    if (vec) {
        const int per_row = g.IX / 16;
        for (int i = tid; i < g.IY * per_row; i += FB_THREADS) {
            const int r = i / per_row, j = i - r * per_row;
            const uint8_t *src = in + (int64_t)clampi(oy + r, 0, h - 1) * in_pitch + ox + 16 * j;
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(src));
            const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
            float4 *dst = reinterpret_cast<float4 *>(I_s + r * g.IX + 16 * j);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // float 2^23 + byte, minus 2^23: the byte's value, exactly
                const float2 lo = __fadd2_rn(f2(__uint_as_float(__byte_perm(wd[q], 0x4B000000u, 0x7640u)),
                                                __uint_as_float(__byte_perm(wd[q], 0x4B000000u, 0x7641u))),
                                             f2(-8388608.f, -8388608.f));
                const float2 hi = __fadd2_rn(f2(__uint_as_float(__byte_perm(wd[q], 0x4B000000u, 0x7642u)),
                                                __uint_as_float(__byte_perm(wd[q], 0x4B000000u, 0x7643u))),
                                             f2(-8388608.f, -8388608.f));
                dst[q] = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
        }
    } else {
        for (int r = warp; r < g.IY; r += FB_WARPS) {
            const uint8_t *row = in + (int64_t)clampi(oy + r, 0, h - 1) * in_pitch;
            for (int c = lane; c < g.IX; c += 32) I_s[r * g.IX + c] = (float)__ldg(row + clampi(ox + c, 0, w - 1));
        }
    }
    __syncthreads();
    // horizontal pass at columns clamp(x0 - 2 + c), rows paired (2p, 2p + 1)
    {
        const int pairs = g.IY / 2;
        auto hpass = [&](int p, int c) {
            const int X = clampi(x0 - 2 + c, 0, w - 1);
            const float *a = I_s + (2 * p) * g.IX + (X - g.R - ox);
            const float *b = a + g.IX;
            const float2 acc = tap_sum2<KS>(fp, [&](int k) { return f2(a[k], b[k]); });
            H_s[(2 * p) * g.SX + c] = acc.x;
            H_s[(2 * p + 1) * g.SX + c] = acc.y;
        };
        for (int p = warp; p < pairs; p += FB_WARPS)
            for (int c = lane; c < FB_W; c += 32) hpass(p, c);
        for (int i = tid; i < pairs * (g.SX - FB_W); i += FB_THREADS) {     // the last SX - 128 columns
            const int p = i / (g.SX - FB_W);
            hpass(p, FB_W + (i - p * (g.SX - FB_W)));
        }
    }
}

// Steps 1-2 for one block up to the smoothed image S (left in region 0).
template <int KS>
__device__ __forceinline__ void smooth_block(const uint8_t *__restrict__ in, int in_pitch, int w, int h,
                                             const FloatParams &fp, const Geometry &g, int x0, int y0,
                                             float *r0, float *r1)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int oy = y0 - g.pady;
    float *I_s = r0, *H_s = r1;
    // horizontal pass; the border is replicated by clamping (rows always,
    // columns only in blocks that reach past the image's left or right edge)
    const bool aligned = ((((uintptr_t)in) | (uintptr_t)in_pitch) & 15) == 0;
    if (KS > 0 && KS <= 29 && aligned && x0 >= 16 && x0 + FB_W + 32 <= w) {
        // inside the image: horizontal pass from registers, lane = row (a row
        // stride of SX = 132 floats keeps the 16-byte stores conflict-free)
        constexpr int NSEG = FB_W / 16;                     // 8 segments of 16 outputs, then 4 more
        const int rblocks = (g.IY + 31) / 32;
        for (int item = warp; item < (NSEG + 1) * rblocks; item += FB_WARPS) {
            const int seg = item % (NSEG + 1), r = 32 * (item / (NSEG + 1)) + lane;
            if (r >= g.IY) continue;
            const uint8_t *row = in + (int64_t)clampi(oy + r, 0, h - 1) * in_pitch;
            if (seg < NSEG) hrow_regs<(KS > 0 ? KS : 3), 16>(row, x0, 16 * seg, fp, H_s + r * g.SX + 16 * seg);
            else hrow_regs<(KS > 0 ? KS : 3), 4>(row, x0, FB_W, fp, H_s + r * g.SX + FB_W);
        }
        __syncthreads();
    } else {
        staged_hpass<KS>(in, in_pitch, w, h, fp, g, x0, y0, I_s, H_s, aligned);
    }
    __syncthreads();
    // vertical pass at rows clamp(y0 - 2 + r), columns paired (2q, 2q + 1):
    // S(clamp(x), clamp(y)) into region 0
    float *S_s = r0;
    {
        const int qn = g.SX / 2;                            // 66 column pairs
        auto vpass = [&](int r, int q) {
            const int Y = clampi(y0 - 2 + r, 0, h - 1);
            const float *src = H_s + (Y - g.R - oy) * g.SX + 2 * q;
            const float2 acc =
                tap_sum2<KS>(fp, [&](int k) { return *reinterpret_cast<const float2 *>(src + k * g.SX); });
            *reinterpret_cast<float2 *>(S_s + r * g.SX + 2 * q) = acc;
        };
        // four output rows per item: where their source rows are consecutive (no
        // clamping) the KS + 3 rows are loaded once and shared
        constexpr int RB = 4;
        const int groups = g.SY / RB;
        for (int item = tid; item < groups * qn; item += FB_THREADS) {
            const int rg = item / qn, q = item - rg * qn, rb = RB * rg;
            const int Ya = clampi(y0 - 2 + rb, 0, h - 1), Yb = clampi(y0 - 2 + rb + RB - 1, 0, h - 1);
            if constexpr (KS > 0) {
                if (Yb - Ya == RB - 1) {
                    const float *src = H_s + (Ya - g.R - oy) * g.SX + 2 * q;
                    float2 win[KS + RB - 1];
#pragma unroll
                    for (int i = 0; i < KS + RB - 1; ++i) win[i] = *reinterpret_cast<const float2 *>(src + i * g.SX);
#pragma unroll
                    for (int o = 0; o < RB; ++o) {
                        float2 acc = f2(fmul(fp.taps[0], win[o].x), fmul(fp.taps[0], win[o].y));
#pragma unroll
                        for (int k = 1; k < KS; ++k)
                            acc = f2(fadd(acc.x, fmul(fp.taps[k], win[o + k].x)),
                                     fadd(acc.y, fmul(fp.taps[k], win[o + k].y)));
                        *reinterpret_cast<float2 *>(S_s + (rb + o) * g.SX + 2 * q) = acc;
                    }
                    continue;
                }
            }
#pragma unroll 1
            for (int o = 0; o < RB; ++o) vpass(rb + o, q);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- pass 1
template <int KS>
__global__ void __launch_bounds__(FB_THREADS, 2)
k1f_max_kernel(const uint8_t *__restrict__ in, int in_pitch, int w, int h, FloatParams fp, float *d_smax)
{
    extern __shared__ __align__(16) float fsm[];
    const Geometry g = geometry(KS > 0 ? KS : fp.ksize);
    float *r0 = fsm, *r1 = fsm + g.region0;
    const int x0 = blockIdx.x * FB_W, y0 = blockIdx.y * FB_H;
    smooth_block<KS>(in, in_pitch, w, h, fp, g, x0, y0, r0, r1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float best = 0.f;
    for (int r = warp; r < FB_H; r += FB_WARPS) {
        if (y0 + r >= h) break;
        for (int q = lane; q < FB_W / 2; q += 32) {
            const int c = 2 * q;                          // pixels x0 + c, x0 + c + 1
            if (x0 + c >= w) break;
            const float2 s2 = strength2_pair(r0, g.SX, r + 2, c + 2);
            best = fmaxf(best, s2.x);
            if (x0 + c + 1 < w) best = fmaxf(best, s2.y);
        }
    }
    __shared__ float red[FB_WARPS];
    for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(tile::FULL, best, o));
    if (lane == 0) red[warp] = best;
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        for (int k = 0; k < FB_WARPS; ++k) m = fmaxf(m, red[k]);
        // non-negative floats order like their bit patterns
        atomicMax(reinterpret_cast<unsigned int *>(d_smax), __float_as_uint(m));
    }
}

// ---------------------------------------------------------------- pass 2
template <int KS>
__global__ void __launch_bounds__(FB_THREADS, 2)
k1f_edges_kernel(const uint8_t *__restrict__ in, int in_pitch, int w, int h, FloatParams fp,
                 const float *__restrict__ d_smax, HystScratch hs, HystImage img)
{
    extern __shared__ __align__(16) float fsm[];
    __shared__ uint32_t cand_s[FB_H][FB_TX], strong_s[FB_H][FB_TX];
    const Geometry g = geometry(KS > 0 ? KS : fp.ksize);
    float *r0 = fsm, *r1 = fsm + g.region0;
    const int x0 = blockIdx.x * FB_W, y0 = blockIdx.y * FB_H;
    smooth_block<KS>(in, in_pitch, w, h, fp, g, x0, y0, r0, r1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // squared strength on the block and its ring (0 outside the image) into region 1
    const float *S_s = r0;
    float *s_s = r1;
    // pairs of columns j = 2 .. FB_W + 1 (S row r + 1 is image row y0 - 1 + r)
    for (int r = warp; r < g.MY; r += FB_WARPS) {
        const int Y = y0 - 1 + r;
        const bool row_in = Y >= 0 && Y < h;
        for (int q = lane; q < FB_W / 2; q += 32) {
            const int j = 2 + 2 * q, X = x0 - 2 + j;
            float2 s2 = f2(0.f, 0.f);
            if (row_in && X < w) {
                s2 = strength2_pair(S_s, g.SX, r + 1, j);
                if (X + 1 >= w) s2.y = 0.f;
            }
            *reinterpret_cast<float2 *>(s_s + r * g.MX + j) = s2;
        }
    }
    // the ring's outer columns j = 1 and j = FB_W + 2
    for (int i = tid; i < 2 * g.MY; i += FB_THREADS) {
        const int r = i >> 1, j = (i & 1) ? FB_W + 2 : 1;
        const int X = x0 - 2 + j, Y = y0 - 1 + r;
        float s = 0.f;
        if (X >= 0 && X < w && Y >= 0 && Y < h) {
            float gx, gy;
            sobel_at(S_s, g.SX, r + 1, j, gx, gy);
            s = strength2(gx, gy);
        }
        s_s[r * g.MX + j] = s;
    }
    __syncthreads();

    // thresholds: fractions of Mmax = sqrt(smax), float products as in the definition
    const float mmax = __fsqrt_rn(*d_smax);
    const float lo_t = fmul(fp.lo_frac, mmax), hi_t = fmul(fp.hi_frac, mmax);
    const float t_min = fminf(lo_t, hi_t);
    // necessary condition for sqrt_rn(s) > t_min: s > t_min^2 (1 - 2^-23); 1e-4 of slack
    const float s_pre = fmul(fmul(t_min, t_min), 0.9999f);

    // Step 3 + thresholds: one (row, tile column) per warp iteration, lane = column
    for (int item = warp; item < FB_H * FB_TX; item += FB_WARPS) {
        const int r = item / FB_TX, tc = item % FB_TX;
        const int mc = 2 + HT * tc + lane, mr = r + 1;      // index in s_s (and S column)
        const float s = s_s[mr * g.MX + mc];
        bool weak = false, strong = false;
        if (s > s_pre) {
            const float m = __fsqrt_rn(s);
            float gx, gy;
            sobel_at(S_s, g.SX, r + 2, mc, gx, gy);
            const float t = 0.41421356f, ax = fabsf(gx), ay = fabsf(gy);
            int dn, dp;                                         // offsets of n- and n+ in s_s
            if (ay < fmul(ax, t)) { dn = -1; dp = 1; }                                  // H
            else if (ax < fmul(ay, t)) { dn = -g.MX; dp = g.MX; }                       // V
            else if ((gx > 0.f && gy > 0.f) || (gx < 0.f && gy < 0.f)) { dn = -g.MX - 1; dp = g.MX + 1; }  // D
            else { dn = g.MX - 1; dp = -g.MX + 1; }             // A: down-left / up-right
            const float mn = __fsqrt_rn(s_s[mr * g.MX + mc + dn]);
            const float mp = __fsqrt_rn(s_s[mr * g.MX + mc + dp]);
            const bool keep = (m > mn) && (m >= mp);
            strong = keep && m > hi_t;
            weak = keep && (m > lo_t || strong);
        }
        const uint32_t wm = __ballot_sync(tile::FULL, weak), sm = __ballot_sync(tile::FULL, strong);
        if (lane == 0) {
            cand_s[r][tc] = wm;
            strong_s[r][tc] = sm;
        }
    }
    __syncthreads();

    // Step 4, tile-local: warp k floods tile k of the block
    const int txl = warp % FB_TX, tyl = warp / FB_TX;
    const int tx = blockIdx.x * FB_TX + txl, ty = blockIdx.y * FB_TY + tyl;
    if (tx < img.ntx && ty < img.nty) {
        const uint32_t cand = cand_s[tyl * HT + lane][txl];
        const uint32_t strong = strong_s[tyl * HT + lane][txl];
        const uint32_t e = tile::flood_tile(strong, cand, lane);
        tile::store_row(img, tx, ty, lane, e);
        tile::finish_tile(hs, img.tile_base + (uint32_t)ty * (uint32_t)img.ntx + (uint32_t)tx, e, cand, lane);
    }
}

size_t fused_smem_bytes(int ksize)
{
    const Geometry g = geometry(ksize);
    return sizeof(float) * ((size_t)g.region0 + (size_t)g.region1);
}

template <int KS>
cudaError_t launch_pair(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp, float *d_smax,
                        const HystScratch *hs, const HystImage *img, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        const int bytes = (int)fused_smem_bytes(KS > 0 ? KS : MAX_KSIZE);
        cudaError_t e = cudaFuncSetAttribute(k1f_max_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k1f_edges_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((w + FB_W - 1) / FB_W, (h + FB_H - 1) / FB_H);
    const size_t smem = fused_smem_bytes(fp.ksize);
    if (!hs) {
        k1f_max_kernel<KS><<<grid, FB_THREADS, smem, s>>>(in, in_pitch, w, h, fp, d_smax);
    } else {
        k1f_edges_kernel<KS><<<grid, FB_THREADS, smem, s>>>(in, in_pitch, w, h, fp, d_smax, *hs, *img);
    }
    return cudaGetLastError();
}

cudaError_t dispatch(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp, float *d_smax,
                     const HystScratch *hs, const HystImage *img, cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    switch (fp.ksize) {
    case 3: return launch_pair<3>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    case 5: return launch_pair<5>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    case 7: return launch_pair<7>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    case 9: return launch_pair<9>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    case 11: return launch_pair<11>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    default: return launch_pair<0>(in, in_pitch, w, h, fp, d_smax, hs, img, s);
    }
}

}  // namespace

cudaError_t launch_k1f_max(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp, float *d_smax,
                           cudaStream_t s)
{
    return dispatch(in, in_pitch, w, h, fp, d_smax, nullptr, nullptr, s);
}

cudaError_t launch_k1f_edges(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp,
                             const float *d_smax, const HystScratch &hs, HystImage img, cudaStream_t s)
{
    return dispatch(in, in_pitch, w, h, fp, const_cast<float *>(d_smax), &hs, &img, s);
}

}  // namespace canny
