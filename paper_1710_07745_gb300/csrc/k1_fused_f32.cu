// k1_fused_f32.cu -- the float32 variant of Steps 1-4 (paper Sec. 2.2.1). The
// thresholds are fractions of the image's largest strength, a grid-wide
// dependency, so the work splits into two passes:
//
//   pass 1 (k1f_strength_kernel): Gaussian -> Sobel -> squared strength
//     s = gx^2 + gy^2 and the gradient's sector for every pixel, written to a
//     float map and a 2-bit sector map, and reduced to the image maximum smax
//     (one atomicMax per CTA);
//   pass 2 (k1f_nms_kernel): on the few pixels that can pass the low threshold,
//     strength M = sqrt(s), suppression against the two neighbours the sector
//     names, double threshold; then the tile flood fill of the hysteresis on
//     32 x 32 tiles and the 0/255 edge bytes, tile border masks and pending
//     bitmaps for the global passes.
//
// Pass 1 reads the input byte and writes 4.25 bytes per pixel; pass 2 reads
// those maps (with a 1-pixel ring) and writes the edge byte. The largest
// strength is Mmax = sqrt(smax) exactly: a correctly rounded square root is
// monotonic, so the largest root is the root of the largest s.
//
// Arithmetic follows the float32 definition operation by operation (no
// contraction except where a product by 2 is exact): horizontal pass then
// vertical pass, taps accumulated from the first, replicate border; Sobel
// columns summed top to bottom; s = (gx*gx) + (gy*gy); M = sqrt_rn(s).
//
// A pass-1 CTA of 256 threads covers a block of 64 rows x 128 columns (2 x 4
// tiles) and stages it in shared memory: the horizontal pass and the smoothed
// image S, and, for blocks at the image's left or right edge, the input (as
// bytes, with a halo of R + 2 rows and R + 2 columns rounded up to 16, R =
// ksize / 2; blocks inside the image run the horizontal pass from registers).
// Buffers alias once they are dead, so a 7-tap kernel needs 73 KB and three
// CTAs fit on an SM. Work is done on pixel pairs that share their
// shared-memory loads (the horizontal pass pairs two rows, the vertical pass
// and Sobel pair two columns); the arithmetic itself is scalar and correctly
// rounded per operation (__fmul_rn / __fadd_rn, and __fmaf_rn only where the
// product by 2 is exact). The Gaussian's products of a pair of independent
// sums come from one two-wide multiply (mul.rn.f32x2, each half rounded like
// __fmul_rn); the sums stay scalar __fadd_rn. A two-wide multiply feeding a
// two-wide add was found to round once, like a fused multiply-add, whatever
// the contraction settings, so the adds are never two-wide.
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
    int region0, region1;      // floats: input bytes then S; horizontal pass
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
    // the staged input is held as bytes (IY x IX of them) in the floats of region 0
    const int a = (g.IY * g.IX + 3) / 4, b = g.SY * g.SX, c = g.IY * g.SX, d = g.MY * g.MX;
    g.region0 = a > b ? a : b;
    g.region1 = c > d ? c : d;
    return g;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 tap2(const FloatParams &fp, int k) { return f2(fp.taps[k], fp.taps[k]); }

// a * b on both halves, each correctly rounded
__device__ __forceinline__ float2 mul2_rn(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)), "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&r);
}
// a + b on both halves as two scalar correctly rounded adds
__device__ __forceinline__ float2 add2_rn(float2 a, float2 b) { return f2(fadd(a.x, b.x), fadd(a.y, b.y)); }

// One Gaussian tap sum on a pair of independent sums:
// taps[0]*v(0) + taps[1]*v(1) + ..., each product and each sum rounded, both
// sums at once with the two-wide operations. KS = 0: run-time ksize.
template <int KS, typename Load>
__device__ __forceinline__ float2 tap_sum2(const FloatParams &fp, Load v)
{
    float2 acc = mul2_rn(tap2(fp, 0), v(0));
    if constexpr (KS > 0) {
#pragma unroll
        for (int k = 1; k < KS; ++k) acc = add2_rn(acc, mul2_rn(tap2(fp, k), v(k)));
    } else {
        for (int k = 1; k < fp.ksize; ++k) acc = add2_rn(acc, mul2_rn(tap2(fp, k), v(k)));
    }
    return acc;
}

__device__ __forceinline__ float strength2(float gx, float gy) { return fadd(fmul(gx, gx), fmul(gy, gy)); }

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
    static_assert(N % 2 == 0 && NOUT % 4 == 0, "outputs in pairs, stores in fours");
    // the inputs as pairs from even offsets, (v[2j], v[2j+1]), and from odd
    // ones, (v[2j+1], v[2j+2]), so that outputs q, q + 1 take both operands of
    // every tap as one pair
    auto raw = [&](int i) { return __uint_as_float(__byte_perm(wd[(LO + i) >> 2], 0x4B000000u, 0x7640u | ((LO + i) & 3))); };
    const float2 bias = f2(-8388608.f, -8388608.f);
    float2 pe[N / 2], po[N / 2 - 1];
#pragma unroll
    for (int j = 0; j < N / 2; ++j) pe[j] = add2_rn(f2(raw(2 * j), raw(2 * j + 1)), bias);
#pragma unroll
    for (int j = 0; j < N / 2 - 1; ++j) po[j] = add2_rn(f2(raw(2 * j + 1), raw(2 * j + 2)), bias);
    float2 out[NOUT / 2];
#pragma unroll
    for (int qp = 0; qp < NOUT / 2; ++qp) {
        float2 acc = mul2_rn(tap2(fp, 0), pe[qp]);
#pragma unroll
        for (int k = 1; k < KS; ++k)
            acc = add2_rn(acc, mul2_rn(tap2(fp, k), (k & 1) ? po[qp + (k >> 1)] : pe[qp + (k >> 1)]));
        out[qp] = acc;
    }
#pragma unroll
    for (int q = 0; q < NOUT; q += 4)
        *reinterpret_cast<float4 *>(dst + q) = make_float4(out[q / 2].x, out[q / 2].y, out[q / 2 + 1].x, out[q / 2 + 1].y);
}

// Step 1's horizontal pass through a staged copy of the input (blocks at the
// image's left or right edge, or inputs without 16-byte alignment): the input
// block is staged as bytes with clamped columns, then H is computed at the
// clamped columns, rows paired.
template <int KS>
__device__ __forceinline__ void staged_hpass(const uint8_t *__restrict__ in, int in_pitch, int w, int h,
                                             const FloatParams &fp, const Geometry &g, int x0, int y0,
                                             uint8_t *I_s, float *H_s, bool aligned)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ox = x0 - g.padx, oy = y0 - g.pady;
    const bool vec = ox >= 0 && ox + g.IX <= w && aligned;
    if (vec) {
        const int per_row = g.IX / 16;
        for (int i = tid; i < g.IY * per_row; i += FB_THREADS) {
            const int r = i / per_row, j = i - r * per_row;
            const uint8_t *src = in + (int64_t)clampi(oy + r, 0, h - 1) * in_pitch + ox + 16 * j;
            *reinterpret_cast<uint4 *>(I_s + r * g.IX + 16 * j) = __ldg(reinterpret_cast<const uint4 *>(src));
        }
    } else {
        for (int r = warp; r < g.IY; r += FB_WARPS) {
            const uint8_t *row = in + (int64_t)clampi(oy + r, 0, h - 1) * in_pitch;
            for (int c = lane; c < g.IX; c += 32) I_s[r * g.IX + c] = __ldg(row + clampi(ox + c, 0, w - 1));
        }
    }
    __syncthreads();
    // horizontal pass at columns clamp(x0 - 2 + c), rows paired (2p, 2p + 1)
    {
        const int pairs = g.IY / 2;
        auto hpass = [&](int p, int c) {
            const int X = clampi(x0 - 2 + c, 0, w - 1);
            const uint8_t *a = I_s + (2 * p) * g.IX + (X - g.R - ox);
            const uint8_t *b = a + g.IX;
            // a byte's value as a float is exact
            const float2 acc = tap_sum2<KS>(fp, [&](int k) { return f2(__uint2float_rn(a[k]), __uint2float_rn(b[k])); });
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
    uint8_t *I_s = reinterpret_cast<uint8_t *>(r0);
    float *H_s = r1;
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
                        float2 acc = mul2_rn(tap2(fp, 0), win[o]);
#pragma unroll
                        for (int k = 1; k < KS; ++k) acc = add2_rn(acc, mul2_rn(tap2(fp, k), win[o + k]));
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

// Sector of the gradient (gx, gy), 2 bits: 0 H (left / right), 1 V (up / down),
// 2 D (up-left / down-right), 3 A (down-left / up-right); tan 22.5 deg as a float.
__device__ __forceinline__ uint32_t sector_of(float gx, float gy)
{
    const float t = 0.41421356f, ax = fabsf(gx), ay = fabsf(gy);
    // the first test that holds decides, as selects rather than branches
    const bool same_sign = (gx > 0.f && gy > 0.f) || (gx < 0.f && gy < 0.f);
    uint32_t code = same_sign ? 2u : 3u;
    code = (ax < fmul(ay, t)) ? 1u : code;
    code = (ay < fmul(ax, t)) ? 0u : code;
    return code;
}

// Sobel (in the definition's order: columns summed top to bottom; a + 2 b
// formed as fma(2, b, a), the same single rounding since 2 b is exact) and
// squared strength of the pixel pair at S entries (r, c), (r, c + 1), c even,
// sharing the loads; their sectors in bits 0-1 and 2-3 of *sec.
__device__ __forceinline__ float2 strength_sector_pair(const float *S, int sx, int r, int c, uint32_t *sec)
{
    const float *u = S + (r - 1) * sx + c - 2, *m = S + r * sx + c - 2, *d = S + (r + 1) * sx + c - 2;
    const float2 u0 = *reinterpret_cast<const float2 *>(u), u1 = *reinterpret_cast<const float2 *>(u + 2),
                 u2 = *reinterpret_cast<const float2 *>(u + 4);
    const float2 m0 = *reinterpret_cast<const float2 *>(m), m1 = *reinterpret_cast<const float2 *>(m + 2),
                 m2 = *reinterpret_cast<const float2 *>(m + 4);
    const float2 d0 = *reinterpret_cast<const float2 *>(d), d1 = *reinterpret_cast<const float2 *>(d + 2),
                 d2 = *reinterpret_cast<const float2 *>(d + 4);
    const float U[4] = {u0.y, u1.x, u1.y, u2.x}, M[4] = {m0.y, m1.x, m1.y, m2.x}, D[4] = {d0.y, d1.x, d1.y, d2.x};
    float out[2];
    uint32_t code = 0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {                      // pixel at column c + i: index 1 + i
        const float right = fadd(__fmaf_rn(2.f, M[2 + i], U[2 + i]), D[2 + i]);
        const float left = fadd(__fmaf_rn(2.f, M[i], U[i]), D[i]);
        const float down = fadd(__fmaf_rn(2.f, D[1 + i], D[i]), D[2 + i]);
        const float up = fadd(__fmaf_rn(2.f, U[1 + i], U[i]), U[2 + i]);
        const float gx = fadd(right, -left), gy = fadd(down, -up);
        out[i] = strength2(gx, gy);
        code |= sector_of(gx, gy) << (2 * i);
    }
    *sec = code;
    return f2(out[0], out[1]);
}

// Layout of the pass-1 maps for a w x h image: whole blocks, mp floats a row
// (a multiple of FB_W) and rows = a multiple of FB_H; the sector map holds
// four pixels a byte (mp / 4 bytes a row). Pixels outside the image hold 0.
struct MapLayout {
    int mp, rows;
};

__host__ __device__ inline MapLayout map_layout(int w, int h)
{
    return MapLayout{(w + FB_W - 1) / FB_W * FB_W, (h + FB_H - 1) / FB_H * FB_H};
}

// ---------------------------------------------------------------- pass 1
// Steps 1-2 and the sector of Step 3 for one block: squared strengths (0
// outside the image) into smap, sectors into sect, block maximum atomicMax'ed
// into *d_smax. With the input staged as bytes a 7- or 9-tap kernel's buffers
// take at most 75 KB, so three CTAs fit on an SM.
template <int KS>
__global__ void __launch_bounds__(FB_THREADS, 3)
k1f_strength_kernel(const uint8_t *__restrict__ in, int in_pitch, int w, int h, FloatParams fp, float *d_smax,
                    float *__restrict__ smap, uint8_t *__restrict__ sect)
{
    extern __shared__ __align__(16) float fsm[];
    const Geometry g = geometry(KS > 0 ? KS : fp.ksize);
    float *r0 = fsm, *r1 = fsm + g.region0;
    const int x0 = blockIdx.x * FB_W, y0 = blockIdx.y * FB_H;
    smooth_block<KS>(in, in_pitch, w, h, fp, g, x0, y0, r0, r1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const MapLayout L = map_layout(w, h);
    float best = 0.f;
    for (int r = warp; r < FB_H; r += FB_WARPS) {
        const int Y = y0 + r;
        for (int q = lane; q < FB_W / 2; q += 32) {
            const int c = 2 * q, X = x0 + c;              // pixels X, X + 1
            uint32_t code;
            float2 s2 = strength_sector_pair(r0, g.SX, r + 2, c + 2, &code);
            if (Y >= h || X >= w) s2.x = 0.f;
            if (Y >= h || X + 1 >= w) s2.y = 0.f;
            best = fmaxf(best, fmaxf(s2.x, s2.y));
            *reinterpret_cast<float2 *>(smap + (size_t)Y * L.mp + X) = s2;
            // lanes 2k and 2k + 1 hold the two pairs of one 4-pixel sector byte
            const uint32_t other = __shfl_xor_sync(tile::FULL, code, 1);
            if ((lane & 1) == 0) sect[(size_t)Y * (L.mp / 4) + (X >> 2)] = (uint8_t)(code | (other << 4));
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
// Step 3 (suppression) and the thresholds on the pass-1 maps, then Step 4's
// tile flood fill: each warp takes one 32 x 32 tile from start to end (its
// strengths with a 1-pixel ring staged in its own shared memory), so warps
// never wait for one another.
constexpr int NMS_T = HT + 2;                // staged rows / columns of a tile with its ring
constexpr int NMS_TILE = NMS_T * NMS_T;
constexpr int NMS_WARPS = 2;                 // tiles (side by side) per CTA: small CTAs free their
                                             // slots soon after their own tiles are done

__global__ void __launch_bounds__(NMS_WARPS * 32)
k1f_nms_kernel(const float *__restrict__ smap, const uint8_t *__restrict__ sect, int w, int h, FloatParams fp,
               const float *__restrict__ d_smax, HystScratch hs, HystImage img)
{
    __shared__ float s_all[NMS_WARPS * NMS_TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = blockIdx.x * NMS_WARPS + warp, ty = blockIdx.y;
    if (tx >= img.ntx || ty >= img.nty) return;                   // warp-uniform; no block barrier follows
    const MapLayout L = map_layout(w, h);
    float *s_s = s_all + warp * NMS_TILE;                          // entry (r, c): row ty*32 - 1 + r, column tx*32 - 1 + c
    const int X0 = tx * HT, Y0 = ty * HT;
    // sectors of tile row `lane` (32 pixels, 2 bits each)
    const uint2 sec_row = __ldg(reinterpret_cast<const uint2 *>(sect + (size_t)(Y0 + lane) * (L.mp / 4) + (X0 >> 2)));
    // the tile's strengths and ring (0 outside the maps): all loads first
    {
        constexpr int NE = (2 * NMS_T + 31) / 32;                   // ring-column entries per lane
        float v[NMS_T], e[NE];
#pragma unroll
        for (int r = 0; r < NMS_T; ++r) {
            const int Y = Y0 - 1 + r;
            v[r] = (Y >= 0 && Y < L.rows) ? __ldg(smap + (size_t)Y * L.mp + X0 + lane) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < NE; ++k) {                                // entry j: row j / 2, left or right column
            const int j = lane + 32 * k, Y = Y0 - 1 + (j >> 1), Xe = (j & 1) ? X0 + HT : X0 - 1;
            e[k] = (j < 2 * NMS_T && Y >= 0 && Y < L.rows && Xe >= 0 && Xe < L.mp)
                       ? __ldg(smap + (size_t)Y * L.mp + Xe) : 0.f;
        }
#pragma unroll
        for (int r = 0; r < NMS_T; ++r) s_s[r * NMS_T + 1 + lane] = v[r];
#pragma unroll
        for (int k = 0; k < NE; ++k) {
            const int j = lane + 32 * k;
            if (j < 2 * NMS_T) s_s[(j >> 1) * NMS_T + ((j & 1) ? NMS_T - 1 : 0)] = e[k];
        }
    }
    __syncwarp();

    // thresholds: fractions of Mmax = sqrt(smax), float products as in the definition
    const float mmax = __fsqrt_rn(*d_smax);
    const float lo_t = fmul(fp.lo_frac, mmax), hi_t = fmul(fp.hi_frac, mmax);
    const float t_min = fminf(lo_t, hi_t);
    // necessary condition for sqrt_rn(s) > t_min: s > t_min^2 (1 - 2^-23); 1e-4 of slack
    const float s_pre = fmul(fmul(t_min, t_min), 0.9999f);

    // row r of the tile per iteration, lane = column; lane r keeps row r's masks
    uint32_t cand = 0, strong = 0;
    for (int r = 0; r < HT; ++r) {
        const int at = (r + 1) * NMS_T + 1 + lane;
        const float s = s_s[at];
        const uint32_t sec_lo = __shfl_sync(tile::FULL, sec_row.x, r);   // row r, columns 0..15
        const uint32_t sec_hi = __shfl_sync(tile::FULL, sec_row.y, r);   // columns 16..31
        bool weak_px = false, strong_px = false;
        if (s > s_pre) {
            const float m = __fsqrt_rn(s);
            const uint32_t sec = ((lane < 16 ? sec_lo : sec_hi) >> (2 * (lane & 15))) & 3u;
            // offsets of n- and n+: H left / right, V up / down, D up-left / down-right,
            // A down-left / up-right
            const int dn = sec == 0 ? -1 : sec == 1 ? -NMS_T : sec == 2 ? -NMS_T - 1 : NMS_T - 1;
            const float mn = __fsqrt_rn(s_s[at + dn]);
            const float mp = __fsqrt_rn(s_s[at - dn]);
            const bool keep = (m > mn) && (m >= mp);
            strong_px = keep && m > hi_t;
            weak_px = keep && (m > lo_t || strong_px);
        }
        const uint32_t wm = __ballot_sync(tile::FULL, weak_px), sm = __ballot_sync(tile::FULL, strong_px);
        if (lane == r) {
            cand = wm;
            strong = sm;
        }
    }

    // Step 4, tile-local
    const uint32_t e = tile::flood_tile(strong, cand, lane);
    tile::store_row(img, tx, ty, lane, e);
    tile::finish_tile(hs, img.tile_base + (uint32_t)ty * (uint32_t)img.ntx + (uint32_t)tx, e, cand, lane);
}

size_t fused_smem_bytes(int ksize)
{
    const Geometry g = geometry(ksize);
    return sizeof(float) * ((size_t)g.region0 + (size_t)g.region1);
}

template <int KS>
cudaError_t launch_strength(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp, float *d_smax,
                            float *smap, uint8_t *sect, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        const int bytes = (int)fused_smem_bytes(KS > 0 ? KS : MAX_KSIZE);
        cudaError_t e =
            cudaFuncSetAttribute(k1f_strength_kernel<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((w + FB_W - 1) / FB_W, (h + FB_H - 1) / FB_H);
    k1f_strength_kernel<KS><<<grid, FB_THREADS, fused_smem_bytes(fp.ksize), s>>>(in, in_pitch, w, h, fp, d_smax,
                                                                                  smap, sect);
    return cudaGetLastError();
}

}  // namespace

size_t k1f_map_bytes(int w, int h)
{
    if (w <= 0 || h <= 0) return 0;
    const MapLayout L = map_layout(w, h);
    return (size_t)L.mp * L.rows * sizeof(float) + (size_t)(L.mp / 4) * L.rows;
}

cudaError_t launch_k1f_strength(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp,
                                float *d_smax, void *maps, cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    const MapLayout L = map_layout(w, h);
    float *smap = static_cast<float *>(maps);
    uint8_t *sect = reinterpret_cast<uint8_t *>(smap + (size_t)L.mp * L.rows);
    switch (fp.ksize) {
    case 3: return launch_strength<3>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    case 5: return launch_strength<5>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    case 7: return launch_strength<7>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    case 9: return launch_strength<9>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    case 11: return launch_strength<11>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    default: return launch_strength<0>(in, in_pitch, w, h, fp, d_smax, smap, sect, s);
    }
}

namespace {
// Strength M = sqrt_rn(s) of every pixel from pass 1's map, and Mmax = sqrt_rn(smax).
__global__ void k1f_strength_out_kernel(const float *__restrict__ smap, int mp, int w, int h, float *__restrict__ mag,
                                        int mag_pitch, const float *d_smax, float *d_max)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x == 0 && y == 0) *d_max = __fsqrt_rn(*d_smax);
    if (x < w && y < h) mag[(int64_t)y * mag_pitch + x] = __fsqrt_rn(smap[(int64_t)y * mp + x]);
}
}  // namespace

cudaError_t launch_k1f_strength_out(const void *maps, int w, int h, float *mag, int mag_pitch, const float *d_smax,
                                    float *d_max, cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    const MapLayout L = map_layout(w, h);
    const dim3 grid((w + 255) / 256, h);
    k1f_strength_out_kernel<<<grid, 256, 0, s>>>(static_cast<const float *>(maps), L.mp, w, h, mag, mag_pitch, d_smax,
                                                 d_max);
    return cudaGetLastError();
}

cudaError_t launch_k1f_nms(const void *maps, int w, int h, const FloatParams &fp, const float *d_smax,
                           const HystScratch &hs, HystImage img, cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    const MapLayout L = map_layout(w, h);
    const float *smap = static_cast<const float *>(maps);
    const uint8_t *sect = reinterpret_cast<const uint8_t *>(smap + (size_t)L.mp * L.rows);
    const dim3 grid(L.mp / (HT * NMS_WARPS), L.rows / HT);
    k1f_nms_kernel<<<grid, NMS_WARPS * 32, 0, s>>>(smap, sect, w, h, fp, d_smax, hs, img);
    return cudaGetLastError();
}

}  // namespace canny
