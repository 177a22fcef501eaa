// k1_fused.cu -- the integer path of Steps 1-4 of the paper's Sec. 2.2.1 in one
// kernel: Gaussian -> Sobel -> strength -> direction sector -> non-maximum
// suppression -> double threshold -> tile-local hysteresis. The image is read
// once and the edge map written once; the class map never leaves the SM.
//
// A CTA is one warp. Its unit of work is a strip of 224 columns x BAND rows
// (BAND = 64, 160 or 256: 7 x BAND/32 hysteresis tiles); lane L handles the 8
// pixels starting at column X0 - 8 + 8L, lanes 1..28 give the output, lanes 0
// and 29 serve halos, lanes 30 and 31 idle along. One image: one CTA per unit.
// A batch: a persistent grid pops units of all images from a device counter.
//
// Phase 1, sliding down the BAND rows (plus a 4-row halo each side):
//   - TMA loads the strip's input rows (256 bytes from X0 - 16) in chunks of
//     3 rows into a 2-stage shared-memory ring, one mbarrier per stage;
//   - the binomial Gaussian runs on pairs of 16-bit lanes (vertical: a cascade
//     of four pairwise sums; horizontal: packed words with the +128 rounding
//     folded in); neighbour lanes trade halo values by shuffles;
//   - the smoothed bytes become floats S (2^23 + S from a byte permute, minus
//     2^23) and Sobel (column sums and row differences) and the squared
//     strength run in packed float2 arithmetic (__ffma2_rn etc.); every value
//     is an integer below 2^24, so the result is exact;
//   - every row's strengths go to a 5-row ring and its smoothed bytes to a
//     6-row ring in shared memory. Only ~2% of pixels exceed the low
//     threshold: one row later their lanes queue one 16-bit entry per such
//     pixel (column, row); after every 3 rows the lanes share the queued
//     pixels (one each), form their Sobel gradients again from the smoothed
//     rows, and run the sector test and the suppression for them alone,
//     setting bits in the strip's weak/strong row bitmasks. A non-candidate
//     neighbour is at most the low threshold, below any candidate, so its
//     stored strength decides nothing.
//   - units away from every image border run a copy of the band loop
//     compiled without the border and row-range tests.
// Shared memory stays at 13.2 KB per CTA and registers at 128 per thread, so
// 16 one-warp CTAs fit on an SM.
// Phase 2: either the class map is written from the bitmasks (canny_classify),
// or the warp runs the tile flood fill of the hysteresis on them and writes
// 255/0 edge bytes plus the tile border masks and pending bitmaps that the
// global passes need.
#include <cuda.h>
#include <string.h>

#include "hyst_tile.cuh"

namespace canny {

namespace {

using tile::FULL;

constexpr int LPX = 8;                  // pixels per lane per row
constexpr int THREADS = 32;             // one warp per CTA
constexpr int OUT_W = 28 * LPX;         // 224 output columns (lanes 1..28) = 7 hysteresis tiles
constexpr int UNROLL = 3;               // period of the 3-row windows
constexpr int CH = UNROLL;              // input rows per TMA chunk (one chunk per unrolled group)
constexpr int STAGES = 2;               // chunks in flight: 6 rows ahead
constexpr int BOX = 256;                // TMA box width: columns X0-16 .. X0+239
constexpr uint32_t CHUNK_BYTES = BOX * CH;
constexpr int RING = 5;                 // rows of strengths kept
constexpr int SRING = 6;                // rows of smoothed bytes kept
constexpr int QCAP = UNROLL * 28 * LPX; // candidate pixels of one 3-row group, at most
constexpr int TILES_X = OUT_W / HT;
constexpr int MW = OUT_W / 32;          // bitmask words per strip row
static_assert((CH * BOX) % 128 == 0, "TMA stage buffers must stay 128-byte aligned");
static_assert(UNROLL <= RING, "ring slots advance by at most one wrap per group");

// Rows per unit. Each unit consumes a whole number of full mbarrier phase
// cycles (NCH a multiple of 2 * STAGES), so a persistent CTA can run unit after
// unit on the same barriers.
template <int BAND>
struct Band {
    static constexpr int ITERS = BAND + 8;          // input rows Y0-4 .. Y0+BAND+3
    static constexpr int NCH = ITERS / CH;          // chunks per unit
    static constexpr int TILES_Y = BAND / HT;
    static_assert(BAND % HT == 0 && ITERS % UNROLL == 0 && NCH % (2 * STAGES) == 0, "bad band height");
};

constexpr uint32_t MAGIC = 0x4B000000u;             // float 2^23
constexpr uint32_t BIAS = 0x00800080u;              // +128 in both 16-bit lanes
constexpr uint32_t WAIT_LIMIT = 1u << 22;           // bounded mbarrier waits

enum { MODE_CLASSMAP = 0, MODE_EDGES = 1 };

template <int BAND>
struct alignas(128) Smem {
    uint8_t in[STAGES][CH * BOX];        // TMA destinations, 128-byte aligned
    float m2[RING][256];                 // strengths of the last rows, by row mod RING
    uint8_t srow[SRING][256];            // smoothed bytes of the last rows, by row mod SRING
    uint16_t queue[QCAP];                // pixel | row in group << 8
    uint32_t cand[BAND][MW];             // class >= 1 (weak or strong), bit = column
    uint32_t strong[BAND][MW];           // class == 2
    uint32_t qcount;
    uint32_t pad;
    unsigned long long full[STAGES];     // mbarriers of the input ring
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(saddr(dst)), "l"(map), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t perm(uint32_t a, uint32_t b, uint32_t sel) { return __byte_perm(a, b, sel); }

// float 2^23 + (byte k of w)
__device__ __forceinline__ float sbyte(uint32_t w, int k)
{
    return __uint_as_float(perm(w, MAGIC, 0x7540u | (uint32_t)k));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }

// 4 bytes of value 0/1 from the low 4 bits of t
__device__ __forceinline__ uint32_t nib01(uint32_t t) { return ((t & 0xFu) * 0x00204081u) & 0x01010101u; }

// Pixel k in [-1, 8] of a row held as pairs p[j] = (x_j, x_{j+4}), p[4] = (x_-1, x_8).
__device__ __forceinline__ float &pix(float2 (&p)[5], int k)
{
    return k < 0 ? p[4].x : (k > 7 ? p[4].y : (k < 4 ? p[k].x : p[k - 4].y));
}

// ---------------------------------------------------------------- candidate suppression
// Step 3 + thresholds for one queued candidate pixel.
// ybase: image row of the group's first queued row, sb: its strength ring slot,
// tb: the smoothed-row ring slot of the row above it (row ybase - 1).
// The pixel's Sobel gradients are computed again from the smoothed rows (the
// same exact integers the stencil formed in floats), with the replicate border
// taken by clamping the neighbour row and column to the image.
template <int BAND, bool INTERIOR>
__device__ __forceinline__ void suppress_pixel(Smem<BAND> &S, uint32_t entry, int sb, int tb, int ybase, int Y0,
                                               int X0, int w, int h, float hi2, uint32_t *err)
{
    const int off = (int)((entry >> 8) & 3u), y = ybase + off, p = (int)(entry & 255u);
    int sl = sb + off;
    if (sl >= RING) sl -= RING;
    const int su = sl == 0 ? RING - 1 : sl - 1, sd = sl == RING - 1 ? 0 : sl + 1;
    int tu = tb + off;
    if (tu >= SRING) tu -= SRING;
    int tc = tu + 1;
    if (tc >= SRING) tc -= SRING;
    int td = tc + 1;
    if (td >= SRING) td -= SRING;
    if (!INTERIOR && y == 0) tu = tc;                  // S(x, -1) = S(x, 0)
    if (!INTERIOR && y == h - 1) td = tc;              // S(x, h) = S(x, h - 1)
    const int c = X0 - LPX + p;                        // image column
    const int pl = INTERIOR || c > 0 ? p - 1 : p, pr = INTERIOR || c < w - 1 ? p + 1 : p;
    const int s_ul = S.srow[tu][pl], s_uc = S.srow[tu][p], s_ur = S.srow[tu][pr];
    const int s_l = S.srow[tc][pl], s_r = S.srow[tc][pr];
    const int s_dl = S.srow[td][pl], s_dc = S.srow[td][p], s_dr = S.srow[td][pr];
    const int gx = (s_ur + 2 * s_r + s_dr) - (s_ul + 2 * s_l + s_dl);
    const int gy = (s_dl + 2 * s_dc + s_dr) - (s_ul + 2 * s_uc + s_ur);
    const float m = S.m2[sl][p];
    // all eight neighbour strengths at once, then pick by sector
    const float l = S.m2[sl][p - 1], r = S.m2[sl][p + 1];
    const float ul = S.m2[su][p - 1], uc = S.m2[su][p], ur = S.m2[su][p + 1];
    const float dl = S.m2[sd][p - 1], dc = S.m2[sd][p], dr = S.m2[sd][p + 1];
    const int ax = abs(gx), ay = abs(gy);
    const bool hz = ay * 32768 < ax * 13573;           // H: left / right
    const bool vt = ax * 32768 < ay * 13573;           // V: up / down
    const bool dg = gx * gy > 0;                       // D: up-left / down-right, else A
    const float mn = hz ? l : vt ? uc : dg ? ul : dl;  // A: down-left / up-right
    const float mp = hz ? r : vt ? dc : dg ? dr : ur;
    if (m > mn && m >= mp) {
        const int col = p - LPX, row = y - Y0;
        if (!CANNY_CHECK(row >= 0 && row < BAND && col >= 0 && col < OUT_W, err)) return;
        atomicOr(&S.cand[row][col >> 5], 1u << (col & 31));
        if (m > hi2) atomicOr(&S.strong[row][col >> 5], 1u << (col & 31));
    }
}

// ---------------------------------------------------------------- phase 1
// INTERIOR: every input row Y0 - 4 .. Y0 + BAND + 4 lies inside the image and
// every lane's columns (and their halos) too, so the border and row-range
// checks are compiled out.
template <bool TMA, int BAND, bool INTERIOR>
__device__ __forceinline__ void stencil_band(const CUtensorMap *tmap, const uint8_t *__restrict__ in,
                                             int in_pitch, int w, int h, IntThresholds t, Smem<BAND> &S, int lane,
                                             int X0, int Y0, uint32_t *err)
{
    constexpr int ITERS = Band<BAND>::ITERS, NCH = Band<BAND>::NCH;
    const int xl = X0 - LPX + LPX * lane;     // image column of the lane's first pixel
    const bool border = !INTERIOR && (xl <= 0 || xl + LPX >= w);
    const bool out_lane = lane >= 1 && lane <= 28 && xl < w;
    const int last = w - 1 - xl;               // index of the lane's last in-image pixel
    const float lo2 = (float)min(t.lo2, 1 << 24), hi2 = (float)min(t.hi2, 1 << 24);
    const bool direct_fast = !TMA && xl >= 0 && xl + LPX <= w &&
                             ((((uintptr_t)in) | (uintptr_t)in_pitch | (uintptr_t)xl) & 7) == 0;
    const int soff = min(LPX + LPX * lane, BOX - LPX);   // lane's bytes in a staged row

    uint32_t rp[4] = {0, 0, 0, 0}, p1[4] = {0, 0, 0, 0}, p2[4] = {0, 0, 0, 0}, p3[4] = {0, 0, 0, 0};
    float2 Sp[3][5];      // S by row slot (row mod 3), pairs (x_j, x_j+4), halo (x_-1, x_8)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int j = 0; j < 5; ++j) Sp[a][j] = f2(0.f, 0.f);
    }
    uint32_t cm_prev = 0;                     // candidate pixels of the previous row
    uint32_t last0 = 0, last1 = 0;            // words of input row h-1, for rows below the image
    uint32_t pf0[UNROLL], pf1[UNROLL];        // direct-load prefetch

    auto direct_load = [&](int y, uint32_t &w0, uint32_t &w1) {
        const uint8_t *row = in + (int64_t)(INTERIOR ? y : clampi(y, 0, h - 1)) * in_pitch;
        if (direct_fast) {
            uint2 v = __ldg(reinterpret_cast<const uint2 *>(row + xl));
            w0 = v.x;
            w1 = v.y;
        } else {
            uint32_t b[LPX];
#pragma unroll
            for (int k = 0; k < LPX; ++k) b[k] = __ldg(row + clampi(xl + k, 0, w - 1));
            w0 = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
            w1 = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
        }
    };
    auto issue_chunk = [&](int c) {           // lane 0 only
        const int slot = c % STAGES;
        mbar_expect_tx(&S.full[slot], CHUNK_BYTES);
        tma_load_2d(&S.in[slot][0], tmap, X0 - 16, Y0 - 4 + c * CH, &S.full[slot]);
    };

    if (TMA) {
        if (lane == 0)
            for (int c = 0; c < STAGES && c < NCH; ++c) issue_chunk(c);
    } else {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) direct_load(Y0 - 4 + u, pf0[u], pf1[u]);
    }
    bool failed = false;
    auto wait_chunk = [&](int c) {
        if (failed) return;
        uint32_t n = 0;
        while (!mbar_try_wait(&S.full[c % STAGES], (uint32_t)(c / STAGES) & 1u))
            if (++n > WAIT_LIMIT) { failed = true; break; }
        if (failed && lane == 0) atomicOr(err, 2u);
    };

    // ring slot (row mod RING) of strength row r = Y0 - 7 + g, kept incrementally,
    // and slot (row mod SRING) of smoothed row Y0 - 6 + g (it alternates: g steps by 3)
    int rsg = (((Y0 - 7) % RING) + RING) % RING;
    int tsg = (((Y0 - 6) % SRING) + SRING) % SRING;
    for (int g = 0; g < ITERS; g += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int i = g + u;
            const int yin = Y0 - 4 + i;          // input row of this iteration
            const int s = yin - 2;               // smoothed row completed now
            const int a = u % 3;                 // slot of row s
            const int am1 = (u + 2) % 3, am2 = (u + 1) % 3;

            // ---- the lane's 8 input bytes of row clamp(yin)
            uint32_t w0, w1;
            if (TMA) {
                const int c = g / CH, off = u, slot = c % STAGES;
                if (off == 0) {
                    wait_chunk(c);
                    if (!INTERIOR && yin < 0) wait_chunk(4 / CH);   // top band: row 0 is in that chunk
                }
                if (!INTERIOR && yin >= h) {
                    w0 = last0;
                    w1 = last1;
                } else {
                    // rows above the image repeat row 0, which sits in chunk 1 (yin = -4..-2) or 0
                    const uint8_t *row = !INTERIOR && yin < 0 ? &S.in[(4 / CH) % STAGES][(4 % CH) * BOX]
                                                              : &S.in[slot][off * BOX];
                    if (!border) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(row + soff);
                        w0 = v.x;
                        w1 = v.y;
                    } else {
                        uint32_t b[LPX];
#pragma unroll
                        for (int k = 0; k < LPX; ++k)
                            b[k] = row[clampi(clampi(xl + k, 0, w - 1) - (X0 - 16), 0, BOX - 1)];
                        w0 = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
                        w1 = b[4] | (b[5] << 8) | (b[6] << 16) | (b[7] << 24);
                    }
                    if (!INTERIOR && yin == h - 1) {
                        last0 = w0;
                        last1 = w1;
                    }
                }
                if (off == CH - 1) {             // chunk consumed: refill its stage
                    __syncwarp();
                    if (lane == 0 && c + STAGES < NCH && !failed) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue_chunk(c + STAGES);
                    }
                }
            } else {
                w0 = pf0[u];
                w1 = pf1[u];
                if (i + UNROLL < ITERS) direct_load(yin + UNROLL, pf0[u], pf1[u]);
            }

            // ---- Step 1: vertical binomial cascade
            uint32_t q[4];
            q[0] = perm(w0, 0, 0x4240u);   // pixels (0, 2)
            q[1] = perm(w0, 0, 0x4341u);   // pixels (1, 3)
            q[2] = perm(w1, 0, 0x4240u);   // pixels (4, 6)
            q[3] = perm(w1, 0, 0x4341u);   // pixels (5, 7)
            uint32_t v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t n1 = rp[k] + q[k];
                const uint32_t n2 = p1[k] + n1;
                const uint32_t n3 = p2[k] + n2;
                v[k] = p3[k] + n3;
                rp[k] = q[k];
                p1[k] = n1;
                p2[k] = n2;
                p3[k] = n3;
            }
            if (i < 4) continue;                 // cascade still filling (warp-uniform)

            // ---- Step 1: horizontal binomial on the packed vertical sums
            const uint32_t Lh = __shfl_up_sync(FULL, perm(v[2], v[3], 0x7632u), 1);   // (V-2, V-1)
            const uint32_t Rh = __shfl_down_sync(FULL, perm(v[0], v[1], 0x5410u), 1); // (V8, V9)
            const uint32_t A = perm(Lh, v[0], 0x5410u);   // (V-2, V0)
            const uint32_t B = perm(Lh, v[1], 0x5432u);   // (V-1, V1)
            const uint32_t C = perm(v[0], v[2], 0x5432u); // (V2, V4)
            const uint32_t D = perm(v[1], v[3], 0x5432u); // (V3, V5)
            const uint32_t F = perm(v[2], Rh, 0x5432u);   // (V6, V8)
            const uint32_t G = perm(v[3], Rh, 0x7632u);   // (V7, V9)
            const uint32_t he0 = A + C + BIAS + 4u * (B + v[1]) + 6u * v[0];   // (h0, h2)
            const uint32_t ho0 = B + D + BIAS + 4u * (v[0] + C) + 6u * v[1];   // (h1, h3)
            const uint32_t he1 = C + F + BIAS + 4u * (D + v[3]) + 6u * v[2];   // (h4, h6)
            const uint32_t ho1 = D + G + BIAS + 4u * (v[2] + F) + 6u * v[3];   // (h5, h7)
            // S as floats: 2^23 + byte from a byte permute, minus 2^23 (exact)
            const float2 unbias = f2(-8388608.f, -8388608.f);
            Sp[a][0] = __fadd2_rn(f2(sbyte(he0, 1), sbyte(he1, 1)), unbias);   // (S0, S4)
            Sp[a][1] = __fadd2_rn(f2(sbyte(ho0, 1), sbyte(ho1, 1)), unbias);   // (S1, S5)
            Sp[a][2] = __fadd2_rn(f2(sbyte(he0, 3), sbyte(he1, 3)), unbias);   // (S2, S6)
            Sp[a][3] = __fadd2_rn(f2(sbyte(ho0, 3), sbyte(ho1, 3)), unbias);   // (S3, S7)
            Sp[a][4] = f2(__shfl_up_sync(FULL, Sp[a][3].y, 1), __shfl_down_sync(FULL, Sp[a][0].x, 1));
            {   // the row's smoothed bytes, for the candidates' gradients
                int ts = tsg + u;
                if (ts >= SRING) ts -= SRING;
                *reinterpret_cast<uint2 *>(&S.srow[ts][LPX * lane]) =
                    make_uint2(perm(he0, ho0, 0x7351u), perm(he1, ho1, 0x7351u));
            }
            if (border) {
                // replicate border on S: S(-1) = S(0), S(x >= w) = S(w - 1)
                if (xl == 0) Sp[a][4].x = Sp[a][0].x;
                if (last < LPX + 1) {
                    float sl = Sp[a][4].x;
#pragma unroll
                    for (int k = -1; k <= LPX; ++k) if (k == last) sl = pix(Sp[a], k);
#pragma unroll
                    for (int k = -1; k <= LPX; ++k) if (k > last) pix(Sp[a], k) = sl;
                }
            }
            if (INTERIOR) {
            } else if (s == 0) {                 // S(-1) = S(0)
#pragma unroll
                for (int j = 0; j < 5; ++j) Sp[am1][j] = Sp[a][j];
            } else if (s >= h) {                 // S(h) = S(h - 1)
#pragma unroll
                for (int j = 0; j < 5; ++j) Sp[a][j] = Sp[am1][j];
            }
            if (i < 6) continue;

            // ---- Step 2: Sobel and strength of row r = s-1 (slots am2, am1, a = rows r-1, r, r+1)
            const int r = s - 1;
            float2 E[5], CS[5];
            const float2 two = f2(2.f, 2.f);
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                E[j] = sub2(Sp[a][j], Sp[am2][j]);                                     // S(r+1) - S(r-1)
                CS[j] = __fadd2_rn(__ffma2_rn(Sp[am1][j], two, Sp[am2][j]), Sp[a][j]);  // column sums (<= 1020)
            }
            float2 gx[4], gy[4], m[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 cl = j > 0 ? CS[j - 1] : f2(CS[4].x, CS[3].x);   // column sum at x-1
                const float2 cr = j < 3 ? CS[j + 1] : f2(CS[0].y, CS[4].y);   // column sum at x+1
                gx[j] = sub2(cr, cl);
                const float2 el = j > 0 ? E[j - 1] : f2(E[4].x, E[3].x);   // E(x-1)
                const float2 er = j < 3 ? E[j + 1] : f2(E[0].y, E[4].y);   // E(x+1)
                gy[j] = __fadd2_rn(__ffma2_rn(E[j], two, el), er);
                m[j] = __ffma2_rn(gx[j], gx[j], __fmul2_rn(gy[j], gy[j]));
            }
            if (!INTERIOR && (r < 0 || r >= h)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) m[j] = f2(0.f, 0.f);
            } else if (border) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (xl + j < 0 || j > last) m[j].x = 0.f;
                    if (xl + j + 4 < 0 || j + 4 > last) m[j].y = 0.f;
                }
            }
            // every row's strengths go to the ring (neighbours of later candidates)
            int rs = rsg + u;
            if (rs >= RING) rs -= RING;
            float4 *mdst = reinterpret_cast<float4 *>(&S.m2[rs][LPX * lane]);
            mdst[0] = make_float4(m[0].x, m[1].x, m[2].x, m[3].x);
            mdst[1] = make_float4(m[0].y, m[1].y, m[2].y, m[3].y);
            // queue the previous row's candidates now that its lower neighbour row exists
            // (row offset u within this group's queued rows Y0 - 8 + g .. Y0 - 6 + g)
            if (cm_prev && r - 1 >= Y0 && r - 1 < Y0 + BAND) {
                uint32_t idx = atomicAdd(&S.qcount, (uint32_t)__popc(cm_prev));
#pragma unroll
                for (int k = 0; k < LPX; ++k)      // static indices keep gprev in registers
                    if ((cm_prev >> k) & 1u)
                        if (CANNY_CHECK(idx < QCAP, err))
                            S.queue[idx++] = (uint16_t)((LPX * lane + k) | (u << 8));
            }
            // which pixels are candidates
            uint32_t cm = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cm |= (m[j].x > lo2 ? 1u : 0u) << j;
                cm |= (m[j].y > lo2 ? 1u : 0u) << (j + 4);
            }
            cm_prev = out_lane ? cm : 0u;
        }
        // ---- Step 3 + thresholds for the queued pixels (their rows +-1 are in the ring)
        __syncwarp();
        const uint32_t n = S.qcount;
        const int sb = rsg == 0 ? RING - 1 : rsg - 1;   // slot of row Y0 - 8 + g
        const int tb = tsg >= 3 ? tsg - 3 : tsg + 3;    // slot of row Y0 - 9 + g
        for (uint32_t j = lane; j < n && CANNY_CHECK(j < QCAP, err); j += 32)
            suppress_pixel<BAND, INTERIOR>(S, S.queue[j], sb, tb, Y0 - 8 + g, Y0, X0, w, h, hi2, err);
        __syncwarp();
        if (lane == 0) S.qcount = 0;
        __syncwarp();
        rsg += UNROLL;
        if (rsg >= RING) rsg -= RING;
        tsg = tsg >= 3 ? tsg - 3 : tsg + 3;
    }
}

// ---------------------------------------------------------------- one unit
// Everything one CTA does for one strip x band of one image.
struct Unit {
    const uint8_t *in;
    int in_pitch, w, h;
    int X0, Y0, sx, sy;        // strip origin, strip and band index
    bool tma;
};

// A unit away from every image border: input rows Y0 - 4 .. Y0 + BAND + 4 and
// the columns of all 32 lanes with their halos (X0 - 16 .. X0 + 247) in the image.
template <int BAND>
__device__ __forceinline__ bool interior_unit(const Unit &U)
{
    return U.X0 >= 16 && U.X0 + 248 <= U.w && U.Y0 >= 4 && U.Y0 + BAND + 4 < U.h;
}

// PATH: 0 = per unit (U.tma), 1 = TMA only, 2 = direct loads only. A kernel that
// holds one path only is compiled for that path alone (no register pressure
// from the other).
enum { PATH_EITHER = 0, PATH_TMA = 1, PATH_DIRECT = 2 };

// SPLIT: interior units take the stencil compiled without border checks. The
// batch kernel, whose units are mostly border units of small images, holds the
// general stencil alone (two copies of the loop in one kernel cost it more in
// instruction fetch than the interior units gain).
template <int BAND, int MODE, int PATH, bool SPLIT>
__device__ __forceinline__ void run_unit(const CUtensorMap *tmap, const Unit &U, IntThresholds t, uint8_t *out,
                                         int out_pitch, const HystScratch &hs, const HystImage &img, uint32_t *err,
                                         Smem<BAND> &S, int lane)
{
    constexpr int TILES_Y = Band<BAND>::TILES_Y;
    for (int k = lane; k < BAND * MW; k += THREADS) {
        (&S.cand[0][0])[k] = 0u;
        (&S.strong[0][0])[k] = 0u;
    }
    if (lane == 0) S.qcount = 0;
    __syncwarp();
    if (PATH == PATH_TMA || (PATH == PATH_EITHER && U.tma)) {
        // the previous unit's reads of the stage buffers are done before TMA reuses them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (PATH != PATH_DIRECT) {
            if (SPLIT && interior_unit<BAND>(U))
                stencil_band<true, BAND, true>(tmap, U.in, U.in_pitch, U.w, U.h, t, S, lane, U.X0, U.Y0, err);
            else
                stencil_band<true, BAND, false>(tmap, U.in, U.in_pitch, U.w, U.h, t, S, lane, U.X0, U.Y0, err);
        }
    } else {
        if constexpr (PATH != PATH_TMA) {
            if (SPLIT && interior_unit<BAND>(U))
                stencil_band<false, BAND, true>(tmap, U.in, U.in_pitch, U.w, U.h, t, S, lane, U.X0, U.Y0, err);
            else
                stencil_band<false, BAND, false>(tmap, U.in, U.in_pitch, U.w, U.h, t, S, lane, U.X0, U.Y0, err);
        }
    }
    __syncwarp();

    if (MODE == MODE_CLASSMAP) {
        // class byte = weak bit + strong bit
        for (int k = lane; k < BAND * MW; k += THREADS) {
            const int row = k / MW, wj = k % MW;
            const int y = U.Y0 + row, x = U.X0 + 32 * wj;
            if (y >= U.h || x >= U.w) continue;
            const uint32_t c = S.cand[row][wj], sgl = S.strong[row][wj];
            uint32_t wd[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) wd[q] = nib01(c >> (4 * q)) + nib01(sgl >> (4 * q));
            uint8_t *dst = out + (int64_t)y * out_pitch + x;
            if (x + 32 <= U.w) {
                tile::store32(dst, wd);
            } else {
                for (int b = 0; b < 32 && x + b < U.w; ++b) dst[b] = (uint8_t)((wd[b >> 2] >> (8 * (b & 3))) & 0xFF);
            }
        }
    } else {
        // Step 4, tile-local: flood fill each of the unit's 7 x BAND/32 tiles from its bitmasks
        for (int tl = 0; tl < TILES_X * TILES_Y; ++tl) {
            const int txl = tl % TILES_X, tyl = tl / TILES_X;
            const int tx = U.sx * TILES_X + txl, ty = U.sy * TILES_Y + tyl;
            if (tx >= img.ntx || ty >= img.nty) continue;         // warp-uniform
            const uint32_t cand = S.cand[tyl * HT + lane][txl];
            const uint32_t strong = S.strong[tyl * HT + lane][txl];
            const uint32_t e = tile::flood_tile(strong, cand, lane);
            tile::store_row(img, tx, ty, lane, e);
            tile::finish_tile(hs, img.tile_base + (uint32_t)ty * (uint32_t)img.ntx + (uint32_t)tx, e, cand, lane);
        }
    }
    __syncwarp();
}

template <int BAND>
__device__ __forceinline__ void init_barriers(Smem<BAND> &S, int lane)
{
    if (lane == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(&S.full[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
}

// ---------------------------------------------------------------- kernels
// One image: one CTA per unit (blockIdx.x = strip, blockIdx.y = band, reordered).
template <int BAND, int MODE, int PATH>
__global__ void __launch_bounds__(THREADS, BAND == 64 ? 16 : 12)
k1_fused_kernel(const __grid_constant__ CUtensorMap tmap, const uint8_t *__restrict__ in, int in_pitch,
                int w, int h, IntThresholds t, uint8_t *__restrict__ out, int out_pitch,
                HystScratch hs, HystImage img, uint32_t *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<BAND> &S = *reinterpret_cast<Smem<BAND> *>(smem_raw);
    const int lane = threadIdx.x;
    init_barriers(S, lane);
    Unit U;
    U.in = in;
    U.in_pitch = in_pitch;
    U.w = w;
    U.h = h;
    U.sx = blockIdx.x;
    // the bottom band row (border units, the slower stencil) starts right after
    // the top one instead of in the last wave: bands 0, nb - 1, 1, 2, ..., nb - 2
    const int nb = (int)gridDim.y, by = (int)blockIdx.y;
    U.sy = by == 0 || nb < 3 ? by : (by == 1 ? nb - 1 : by - 1);
    U.X0 = U.sx * OUT_W;
    U.Y0 = U.sy * BAND;
    U.tma = PATH == PATH_TMA;
    run_unit<BAND, MODE, PATH, true>(&tmap, U, t, out, out_pitch, hs, img, err, S, lane);
}

// One (image, strip, band) unit of a batch.
template <int BAND, int PATH>
__device__ __forceinline__ void batch_unit(const BatchImage *__restrict__ imgs, const CUtensorMap *__restrict__ tmaps,
                                           int nimg, uint32_t unit, IntThresholds t, const HystScratch &hs,
                                           Smem<BAND> &S, int lane)
{
    int lo = 0, hi = nimg - 1;                     // last image whose units start at or before unit
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].unit_base <= unit) lo = mid;
        else hi = mid - 1;
    }
    const BatchImage &B = imgs[lo];
    const uint32_t local = unit - B.unit_base;
    Unit U;
    U.in = B.in;
    U.in_pitch = B.in_pitch;
    U.w = B.img.w;
    U.h = B.img.h;
    U.sx = (int)(local % (uint32_t)B.nsx);
    U.sy = (int)(local / (uint32_t)B.nsx);
    U.X0 = U.sx * OUT_W;
    U.Y0 = U.sy * BAND;
    U.tma = PATH == PATH_TMA || B.tma != 0;
    const HystImage img = B.img;
    if (U.tma && lane == 0) {
        // the descriptor was rewritten in global memory since the TMA unit may
        // last have cached one at this address: order that write before its use
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&tmaps[lo]) : "memory");
    }
    __syncwarp();
    run_unit<BAND, MODE_EDGES, PATH, false>(&tmaps[lo], U, t, img.map, img.pitch, hs, img, &hs.state->error, S, lane);
}

// A batch. PERSIST: a persistent grid pops units from a counter; otherwise the
// grid has one CTA per unit (set per launch) and the hardware schedules them.
// PATH_TMA when every input is TMA-readable, else PATH_EITHER (chosen per image).
template <int BAND, int PATH, bool PERSIST>
__global__ void __launch_bounds__(THREADS, BAND == 64 ? 16 : 12)
k1_fused_batch_kernel(const BatchImage *__restrict__ imgs, const CUtensorMap *__restrict__ tmaps,
                      BatchHeader *hdr, IntThresholds t, HystScratch hs)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<BAND> &S = *reinterpret_cast<Smem<BAND> *>(smem_raw);
    const int lane = threadIdx.x;
    const uint32_t total = hdr->total_units;
    const int nimg = (int)hdr->nimg;
    if constexpr (!PERSIST) {
        if (blockIdx.x >= total) return;
        init_barriers(S, lane);
        batch_unit<BAND, PATH>(imgs, tmaps, nimg, blockIdx.x, t, hs, S, lane);
    } else {
        init_barriers(S, lane);
        for (;;) {
            uint32_t unit = 0;
            if (lane == 0) unit = atomicAdd(&hdr->next_unit, 1u);
            unit = __shfl_sync(FULL, unit, 0);
            if (unit >= total) break;
            batch_unit<BAND, PATH>(imgs, tmaps, nimg, unit, t, hs, S, lane);
        }
    }
}

template <int BAND, int MODE>
cudaError_t launch_single(const CUtensorMap &tmap, bool tma, const uint8_t *in, int in_pitch, int w, int h,
                          IntThresholds t, uint8_t *out, int out_pitch, const HystScratch &hs, const HystImage &img,
                          uint32_t *err, cudaStream_t s)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k1_fused_kernel<BAND, MODE, PATH_TMA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<BAND>));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k1_fused_kernel<BAND, MODE, PATH_DIRECT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<BAND>));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((w + OUT_W - 1) / OUT_W, (h + BAND - 1) / BAND);
    if (tma)
        k1_fused_kernel<BAND, MODE, PATH_TMA><<<grid, THREADS, sizeof(Smem<BAND>), s>>>(
            tmap, in, in_pitch, w, h, t, out, out_pitch, hs, img, err);
    else
        k1_fused_kernel<BAND, MODE, PATH_DIRECT><<<grid, THREADS, sizeof(Smem<BAND>), s>>>(
            tmap, in, in_pitch, w, h, t, out, out_pitch, hs, img, err);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_any(int band, const uint8_t *in, int in_pitch, int w, int h, IntThresholds t, uint8_t *out,
                       int out_pitch, const HystScratch &hs, const HystImage &img, uint32_t *err, cudaStream_t s)
{
    CUtensorMap tmap;
    memset(&tmap, 0, sizeof(tmap));
    const bool tma = encode_u8_map(&tmap, in, w, h, in_pitch, BOX, CH);
    switch (band) {
    case 160: return launch_single<160, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    case 256: return launch_single<256, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    default: return launch_single<64, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    }
}

}  // namespace

bool k1_band_supported(int band) { return band == 64 || band == 160 || band == 256; }

int k1_units(int w, int h, int band)
{
    if (w <= 0 || h <= 0) return 0;
    return ((w + OUT_W - 1) / OUT_W) * ((h + band - 1) / band);
}

int k1_strip_width() { return OUT_W; }

cudaError_t launch_k1_classify_u8(const uint8_t *in, int in_pitch, uint8_t *cls, int cls_pitch, int w, int h,
                                  IntThresholds t, uint32_t *err, cudaStream_t s, int band)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    HystScratch none = {};
    HystImage img = {};
    return launch_any<MODE_CLASSMAP>(band, in, in_pitch, w, h, t, cls, cls_pitch, none, img, err, s);
}

cudaError_t launch_k1_edges_u8(const uint8_t *in, int in_pitch, int w, int h, IntThresholds t,
                               const HystScratch &hs, HystImage img, cudaStream_t s, int band)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    return launch_any<MODE_EDGES>(band, in, in_pitch, w, h, t, img.map, img.pitch, hs, img, &hs.state->error, s);
}

// Kernel node parameters of the batch kernel; grid: CTAs (persistent) or units.
template <int BAND, int PATH, bool PERSIST>
cudaError_t batch_node_params(const BatchImage *const &imgs, const CUtensorMap *const &tmaps, BatchHeader *const &hdr,
                              const IntThresholds &t, const HystScratch &hs, unsigned grid, void **args,
                              cudaKernelNodeParams *kp)
{
    cudaError_t e = cudaFuncSetAttribute(k1_fused_batch_kernel<BAND, PATH, PERSIST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<BAND>));
    if (e != cudaSuccess) return e;
    args[0] = (void *)&imgs;
    args[1] = (void *)&tmaps;
    args[2] = (void *)&hdr;
    args[3] = (void *)&t;
    args[4] = (void *)&hs;
    *kp = cudaKernelNodeParams{};
    kp->func = (void *)k1_fused_batch_kernel<BAND, PATH, PERSIST>;
    kp->gridDim = dim3(grid > 0 ? grid : 1u);
    kp->blockDim = dim3(THREADS);
    kp->sharedMemBytes = sizeof(Smem<BAND>);
    kp->kernelParams = args;
    return cudaSuccess;
}

template <int BAND>
cudaError_t batch_params_band(bool tma_only, bool persist, const BatchImage *const &imgs,
                              const CUtensorMap *const &tmaps, BatchHeader *const &hdr, const IntThresholds &t,
                              const HystScratch &hs, unsigned grid, void **args, cudaKernelNodeParams *kp)
{
    if (tma_only)
        return persist ? batch_node_params<BAND, PATH_TMA, true>(imgs, tmaps, hdr, t, hs, grid, args, kp)
                       : batch_node_params<BAND, PATH_TMA, false>(imgs, tmaps, hdr, t, hs, grid, args, kp);
    return persist ? batch_node_params<BAND, PATH_EITHER, true>(imgs, tmaps, hdr, t, hs, grid, args, kp)
                   : batch_node_params<BAND, PATH_EITHER, false>(imgs, tmaps, hdr, t, hs, grid, args, kp);
}

cudaError_t batch_params(int band, bool tma_only, bool persist, const BatchImage *const &imgs,
                         const CUtensorMap *const &tmaps, BatchHeader *const &hdr, const IntThresholds &t,
                         const HystScratch &hs, unsigned grid, void **args, cudaKernelNodeParams *kp)
{
    switch (band) {
    case 160: return batch_params_band<160>(tma_only, persist, imgs, tmaps, hdr, t, hs, grid, args, kp);
    case 256: return batch_params_band<256>(tma_only, persist, imgs, tmaps, hdr, t, hs, grid, args, kp);
    default: return batch_params_band<64>(tma_only, persist, imgs, tmaps, hdr, t, hs, grid, args, kp);
    }
}

cudaError_t k1_add_batch_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, int band, bool tma_only,
                              const BatchImage *imgs, const CUtensorMap *tmaps, BatchHeader *hdr, IntThresholds t,
                              const HystScratch &hs, int ctas, cudaGraphNode_t *out)
{
    void *args[5];
    cudaKernelNodeParams kp;
    cudaError_t e = batch_params(band, tma_only, ctas > 0, imgs, tmaps, hdr, t, hs, (unsigned)(ctas > 0 ? ctas : 1),
                                 args, &kp);
    if (e != cudaSuccess) return e;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

cudaError_t k1_set_batch_units(cudaGraphExec_t exec, cudaGraphNode_t node, int band, bool tma_only,
                               const BatchImage *imgs, const CUtensorMap *tmaps, BatchHeader *hdr, IntThresholds t,
                               const HystScratch &hs, uint32_t units)
{
    void *args[5];
    cudaKernelNodeParams kp;
    cudaError_t e = batch_params(band, tma_only, false, imgs, tmaps, hdr, t, hs, units, args, &kp);
    if (e != cudaSuccess) return e;
    return cudaGraphExecKernelNodeSetParams(exec, node, &kp);
}

bool encode_k1_map(void *tmap_out, const uint8_t *in, int w, int h, int in_pitch)
{
    return encode_u8_map(tmap_out, in, w, h, in_pitch, BOX, CH);
}

}  // namespace canny
