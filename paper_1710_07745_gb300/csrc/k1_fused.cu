// k1_fused.cu -- the integer path of Steps 1-3 and Step 4's double threshold
// of the paper's Sec. 2.2.1 in one kernel: Gaussian -> Sobel -> strength ->
// direction sector -> non-maximum suppression -> double threshold, written as
// two bits per pixel (weak-or-strong, strong) into the tile scratch; the tile
// fill kernel (tile_fill.cu), launched right after it, runs the tile-local
// hysteresis and writes the edge map. The image is read once and the edge map
// written once; the class map never exists as bytes.
//
// A CTA is one warp. Its unit of work is a strip of 480 columns x BAND rows
// (15 x BAND/32 hysteresis tiles). Lane L owns the 16 pixels starting at
// column X0 - 16 + 16 L; lanes 1..30 give the output, lanes 0 and 31 supply
// the halo columns. The warp slides down the BAND rows plus a 4-row halo on
// each side, three rows per group:
//   - TMA stages the strip's input rows (512 bytes from X0 - 16, as two
//     256-byte boxes) three rows per chunk into a 2-stage ring, one mbarrier
//     per stage;
//   - Step 1, binomial 5x5: a lane's 16 bytes become eight 16-bit pairs
//     E_k = (x_4k, x_4k+2), O_k = (x_4k+1, x_4k+3); the vertical pass is
//     (1,2,1) applied twice, the horizontal pass weights shifted pairs (+128
//     rounding folded in), all in integer SWAR. Every row-to-row state (the
//     two vertical stages, Sobel's Dx and T) spans two rows, so with three
//     rows per group the registers rotate without copies;
//   - Step 2, Sobel: the smoothed bytes S become fp16 pairs 1024 + S by one
//     byte permute; every Sobel sum is an integer of magnitude below 2048,
//     which fp16 holds exactly, so Gx and Gy are exact;
//   - candidates: Gx^2 + Gy^2 is compared with the low threshold in fp16
//     with a margin that makes the test a necessary condition (a pixel above
//     the threshold is always flagged; a few below it may be), giving 16
//     flags per lane and row;
//   - every row's exact Gx, Gy go to a 5-row shared ring; after each group the
//     warp deals the flagged pixels of three rows out to its lanes (a prefix
//     sum over the lanes' flag counts), and each lane runs the exact Step 3
//     for its pixel: fp32 strength (exact), the Q15 sector test, suppression
//     against the two neighbours its sector names, and the Step 4
//     thresholds, setting bits in the tile row's weak/strong bitmasks;
//   - after every 32 rows the warp writes the tile row's class bitmasks, 64
//     words per tile (rows 0..31 weak-or-strong, then rows 0..31 strong), for
//     the tile fill (or, for canny_classify, the class bytes).
// Units away from every image border run a copy of the band loop compiled
// without the border and row-range tests.
#include <cuda.h>
#include <cuda_fp16.h>
#include <string.h>

#include "hyst_tile.cuh"

namespace canny {

namespace {

using tile::FULL;

constexpr int LPX = 16;                 // pixels per lane per row
constexpr int THREADS = 32;             // one warp per CTA
constexpr int OUT_LANES = 30;           // lanes 1..30 give the output
constexpr int OUT_W = OUT_LANES * LPX;  // 480 output columns = 15 hysteresis tiles
constexpr int TILES_X = OUT_W / HT;
constexpr int ROWB = THREADS * LPX;     // 512 staged bytes per row: columns X0-16 .. X0+495
constexpr int BOX = 256;                // TMA box width (the hardware limit): two boxes per row
constexpr int U = 3;                    // rows per group = input rows per TMA chunk
constexpr int CH = U;
constexpr int STAGES = 2;               // chunks in flight: 6 rows ahead
constexpr int GRING = U + 2;            // gradient rows kept: a group's candidate rows +-1
constexpr int CROWS = HT + U - 1;       // rows of class bitmasks: a tile row plus a group's overhang
constexpr int GHALF = THREADS * 16;     // bytes of one gradient half-row (E or O pairs of all lanes)
constexpr int GROW = 4 * GHALF;         // one gradient row: Gx E, Gx O, Gy E, Gy O
constexpr uint32_t CHUNK_BYTES = ROWB * CH;
static_assert(OUT_W % HT == 0, "strips hold whole tiles");

// Rows per unit: input rows Y0-4 .. Y0+BAND+3 in groups of U (rounded up to a
// whole group; the extra rows' results are not used).
template <int BAND>
struct Band {
    static constexpr int ITERS = (BAND + 8 + U - 1) / U * U;
    static constexpr int GROUPS = ITERS / U;
    static constexpr int TILES_Y = BAND / HT;
    static_assert(BAND % HT == 0 && ITERS % U == 0 && GROUPS % STAGES == 0, "bad band height");
};

constexpr uint32_t BIAS = 0x00800080u;              // +128 in both 16-bit lanes
constexpr uint32_t H1024 = 0x64006400u;             // fp16 1024 in both halves (exponent byte 0x64)
constexpr uint32_t HTWO = 0x40004000u;              // fp16 2.0
constexpr uint32_t HM3072 = 0xEA00EA00u;            // fp16 -3072

enum { MODE_CLASSMAP = 0, MODE_EDGES = 1 };

struct Smem {                            // at the 128-byte aligned start of dynamic shared memory
    uint8_t in[STAGES][2][CH][BOX];      // TMA destinations: [stage][box][row][column]
    uint8_t g[GRING][GROW];              // exact Gx, Gy (fp16) of the last rows, by row mod GRING
    uint32_t cand[CROWS][TILES_X];       // class >= 1 by (row - Y0) mod CROWS, bit = column
    uint32_t strong[CROWS][TILES_X];     // class == 2
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

// fp16x2 arithmetic on raw bits, round to nearest (every use here is exact
// except the candidate test, whose margin covers its rounding); the intrinsics
// let constant operands be encoded as immediates
__device__ __forceinline__ __half2 as_h2(uint32_t u)
{
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}
__device__ __forceinline__ uint32_t as_u32(__half2 h)
{
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ uint32_t hadd2(uint32_t a, uint32_t b) { return as_u32(__hadd2(as_h2(a), as_h2(b))); }
__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) { return as_u32(__hsub2(as_h2(a), as_h2(b))); }
__device__ __forceinline__ uint32_t hfma2(uint32_t a, uint32_t b, uint32_t c)
{
    return as_u32(__hfma2(as_h2(a), as_h2(b), as_h2(c)));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// 4 bytes of value 0/1 from the low 4 bits of t
__device__ __forceinline__ uint32_t nib01(uint32_t t) { return ((t & 0xFu) * 0x00204081u) & 0x01010101u; }

// Half p (0..15) of a lane's pixels held as E_k = (4k, 4k+2), O_k = (4k+1, 4k+3).
__device__ __forceinline__ uint32_t get_px(const uint32_t (&E)[4], const uint32_t (&O)[4], int p)
{
    const uint32_t w = (p & 1) ? O[p >> 2] : E[p >> 2];
    return (p & 2) ? (w >> 16) : (w & 0xFFFFu);
}
__device__ __forceinline__ void set_px(uint32_t (&E)[4], uint32_t (&O)[4], int p, uint32_t v)
{
    uint32_t &w = (p & 1) ? O[p >> 2] : E[p >> 2];
    w = (p & 2) ? ((w & 0xFFFFu) | (v << 16)) : ((w & 0xFFFF0000u) | v);
}

// Position of the k-th (0-based) set bit of m; m's set bits lie in bits 4..7 of its bytes.
__device__ __forceinline__ uint32_t nth_flag(uint32_t m, uint32_t k)
{
    uint32_t pos = 0, c = __popc(m & 0xFFFFu);
    if (k >= c) { k -= c; m >>= 16; pos = 16; }
    c = __popc(m & 0xFFu);
    if (k >= c) { k -= c; m >>= 8; pos += 8; }
    m >>= 4;
    pos += 4;
    c = __popc(m & 0x3u);
    if (k >= c) { k -= c; m >>= 2; pos += 2; }
    if (k >= (m & 1u)) pos += 1;
    return pos;
}

// Lane-local pixel (0..15) of flag bit b: bit 7 - q of byte B of the flag word
// is the flag of pixel 4q + B.
__device__ __forceinline__ int flag_px(uint32_t b) { return 4 * (7 - (int)(b & 7u)) + (int)(b >> 3); }

// Byte offset, inside a gradient row, of the Gx value of staged column col (0..511):
// lane col / 16 at 16 col / 16 bytes, pair col / 4 mod 4 at 4 times that, high
// half if bit 1 of col is set, the O half-row (+GHALF) if bit 0 is set; together
// that is col with bit 0 moved to bit 9.
__device__ __forceinline__ int gcol_off(int col) { return (col & ~1) + (col & 1) * GHALF; }

__device__ __forceinline__ float gload(const uint8_t *p)
{
    return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short *>(p)));
}

// Exact Gx^2 + Gy^2 at a gradient-row byte offset (0 outside the image).
__device__ __forceinline__ float gstrength(const uint8_t *p)
{
    const float x = gload(p), y = gload(p + 2 * GHALF);
    return fmaf(x, x, y * y);
}

// ---------------------------------------------------------------- Step 3 for one flagged pixel
// rowc, rowu, rowd: gradient rows of the pixel's row and the rows above and below;
// col: staged column (lanes 1..30). The flag is a necessary condition; the exact
// strength decides here.
__device__ __forceinline__ void suppress_pixel(Smem &S, int col, const uint8_t *rowc, const uint8_t *rowu,
                                               const uint8_t *rowd, int trow, float lo2, float hi2, uint32_t *err)
{
    const int off = gcol_off(col);
    const float gx = gload(rowc + off), gy = gload(rowc + off + 2 * GHALF);
    const float m = fmaf(gx, gx, gy * gy);             // exact: integers below 2^24
    if (!(m > lo2)) return;
    const float ax = fabsf(gx), ay = fabsf(gy);
    const bool hz = ay * 32768.f < ax * 13573.f;       // H: left / right (both products exact)
    const bool vt = ax * 32768.f < ay * 13573.f;       // V: up / down
    const bool dg = gx * gy > 0.f;                     // D: up-left / down-right, else A: down-left / up-right
    const int dxn = vt ? 0 : -1;                       // negative-side neighbour (dxn, dyn), positive (-dxn, -dyn)
    const uint8_t *rn = hz ? rowc : (vt || dg ? rowu : rowd);
    const uint8_t *rp = hz ? rowc : (vt || dg ? rowd : rowu);
    const float mn = gstrength(rn + gcol_off(col + dxn));
    const float mp = gstrength(rp + gcol_off(col - dxn));
    if (m > mn && m >= mp) {
        const int oc = col - LPX;                      // output column in the strip
        if (!CANNY_CHECK(oc >= 0 && oc < OUT_W && trow >= 0 && trow < CROWS, err)) return;
        atomicOr(&S.cand[trow][oc >> 5], 1u << (oc & 31));
        if (m > hi2) atomicOr(&S.strong[trow][oc >> 5], 1u << (oc & 31));
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

// Where a unit's results go.
struct Out {
    uint8_t *map;              // class map (MODE_CLASSMAP) or edge map
    int pitch;
    HystScratch hs;
    HystImage img;
};

// The tile row t (32 rows) of the unit is classified: flood its 15 tiles and write
// edges and tile state, or write the class bytes; then clear the bitmask rows.
// Row y of the tile row sits in bitmask row (32 t + y) mod CROWS.
template <int BAND, int MODE>
__device__ __forceinline__ void finish_tile_row(Smem &S, const Unit &U_, const Out &O, int t, int lane)
{
    __syncwarp();
    const int brow = (HT * t + lane) % CROWS;
    if (MODE == MODE_CLASSMAP) {
        const int y = U_.Y0 + t * HT + lane;
#pragma unroll 1
        for (int txl = 0; txl < TILES_X; ++txl) {
            const int x = U_.X0 + HT * txl;
            const uint32_t c = S.cand[brow][txl], sg = S.strong[brow][txl];
            S.cand[brow][txl] = 0u;
            S.strong[brow][txl] = 0u;
            if (y >= U_.h || x >= U_.w) continue;
            uint32_t wd[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) wd[q] = nib01(c >> (4 * q)) + nib01(sg >> (4 * q));
            uint8_t *dst = O.map + (int64_t)y * O.pitch + x;
            if (x + 32 <= U_.w) {
                tile::store32(dst, wd);
            } else {
                for (int b = 0; b < 32 && x + b < U_.w; ++b) dst[b] = (uint8_t)((wd[b >> 2] >> (8 * (b & 3))) & 0xFF);
            }
        }
    } else {
        // the tile row's class bits go to the tile fill: rows of class >= 1, then rows of class 2
        constexpr int TILES_Y = Band<BAND>::TILES_Y;
        const HystImage &im = O.img;
        const int ty = U_.sy * TILES_Y + t;
#pragma unroll 1
        for (int txl = 0; txl < TILES_X; ++txl) {
            const int tx = U_.sx * TILES_X + txl;
            const uint32_t c = S.cand[brow][txl], sg = S.strong[brow][txl];
            S.cand[brow][txl] = 0u;
            S.strong[brow][txl] = 0u;
            if (tx >= im.ntx || ty >= im.nty) continue;                 // warp-uniform
            const uint32_t tid = im.tile_base + (uint32_t)ty * (uint32_t)im.ntx + (uint32_t)tx;
            if (!CANNY_CHECK(tid < O.hs.max_tiles, &O.hs.state->error)) continue;
            uint32_t *bt = O.hs.bits + (size_t)tid * 2 * HT;
            bt[lane] = c;
            bt[HT + lane] = sg;
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- the band loop
// INTERIOR: every input row Y0 - 4 .. Y0 + BAND + 3 lies inside the image and
// every lane's columns too, so the border and row-range checks are compiled out.
template <bool TMA, int BAND, bool INTERIOR, int MODE>
__device__ __forceinline__ void stencil_band(const CUtensorMap *tmap, const Unit &U_, IntThresholds t, const Out &O,
                                             Smem &S, int lane, uint32_t pbase, uint32_t *err)
{
    constexpr int GROUPS = Band<BAND>::GROUPS;
    const int w = U_.w, h = U_.h, X0 = U_.X0, Y0 = U_.Y0;
    const int xl = X0 - LPX + LPX * lane;       // image column of the lane's first pixel
    const bool border = !INTERIOR && (xl < 0 || xl + LPX > w);
    // some lane of the warp is at an image border: the per-lane border work runs
    // behind this warp-uniform test, so units away from the borders skip it
    const bool wborder = !INTERIOR && __any_sync(FULL, border);
    const bool out_lane = lane >= 1 && lane <= OUT_LANES;
    const int e_last = w - 1 - xl;               // lane pixel holding column w - 1 (if 0..15)
    const float lo2 = (float)min(t.lo2, 1 << 24), hi2 = (float)min(t.hi2, 1 << 24);
    // candidate test threshold: largest fp16 at most lo2 (1 - 2^-9) - 1, in [0.5, 65504]
    uint32_t negL;
    {
        const float L = fminf(fmaxf((float)t.lo2 * (1.f - 1.f / 512.f) - 1.f, 0.5f), 65504.f);
        const uint32_t hb = (uint32_t)__half_as_ushort(__float2half_rd(L)) | 0x8000u;   // -L'
        negL = hb | (hb << 16);
    }

    // Row state as 3-slot rings indexed by iteration mod 3 (= u: a group is 3 rows),
    // so no value is ever copied: input rows (pairs E_0..3, O_0..3), first-stage
    // vertical sums a, and Sobel's Dx and T of the smoothed rows.
    static_assert(U == 3, "the row rings below have 3 slots");
    uint32_t rq[3][8], ra[3][8], dx[3][8], tb[3][8];
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int j = 0; j < 8; ++j) rq[z][j] = ra[z][j] = dx[z][j] = tb[z][j] = 0u;
    uint32_t last[4] = {0u, 0u, 0u, 0u};         // words of input row h-1, for rows below the image
    uint32_t mk[U] = {};                         // flag words of a group's candidate rows
    uint32_t carry = 0u;
    int next_tile = 0;                           // next tile row to finish

    auto issue_chunk = [&](int c) {              // lane 0 only
        const int slot = c % STAGES;
        const int y = Y0 - 4 + c * CH;
        mbar_expect_tx(&S.full[slot], CHUNK_BYTES);
        tma_load_2d(&S.in[slot][0][0][0], tmap, X0 - LPX, y, &S.full[slot]);
        tma_load_2d(&S.in[slot][1][0][0], tmap, X0 - LPX + BOX, y, &S.full[slot]);
    };
    bool failed = false;
    auto wait_chunk = [&](int c) {
        if (failed) return;
        const uint32_t parity = ((uint32_t)(c / STAGES) + pbase) & 1u;
        if (mbar_try_wait(&S.full[c % STAGES], parity)) return;
        // bounded by time: a TMA load that has not landed in a second has failed
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(&S.full[c % STAGES], parity))
            if (globaltimer_ns() - t0 > WAIT_TIMEOUT_NS) { failed = true; break; }
        if (failed && lane == 0) atomicOr(err, 2u);
    };
    if (TMA && lane == 0)
        for (int c = 0; c < STAGES && c < GROUPS; ++c) issue_chunk(c);

    // rows above the image repeat row 0: input row index 4 = chunk 4 / CH, row 4 % CH
    constexpr int ROW0_CHUNK = 4 / CH, ROW0_OFF = 4 % CH;
    static_assert(ROW0_CHUNK < STAGES, "row 0 of the top band must be in flight with chunk 0");
    int gsl = 0;                                  // gradient-ring slot of the next Sobel row
#pragma unroll 1
    for (int g = 0; g < GROUPS; ++g) {
        if (TMA) {
            wait_chunk(g);
            if (!INTERIOR && Y0 == 0 && g < ROW0_CHUNK) wait_chunk(ROW0_CHUNK);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = g * U + u;
            const int yin = Y0 - 4 + i;           // input row of this iteration
            const int s = yin - 2;                // smoothed row completed now
            const int r = s - 1;                  // Sobel row completed now

            // ---- the lane's 16 input bytes of row clamp(yin)
            uint32_t wd[4];
            if (!INTERIOR && yin >= h) {
#pragma unroll
                for (int k = 0; k < 4; ++k) wd[k] = last[k];
            } else if (TMA) {
                const bool above = !INTERIOR && yin < 0;
                const int slot = above ? ROW0_CHUNK % STAGES : g % STAGES, ru = above ? ROW0_OFF : u;
                if (!wborder || !border) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(&S.in[slot][lane >> 4][ru][(lane & 15) * LPX]);
                    wd[0] = v.x; wd[1] = v.y; wd[2] = v.z; wd[3] = v.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint32_t b[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int col = clampi(xl + 4 * k + e, 0, w - 1) - (X0 - LPX);
                            b[e] = S.in[slot][col >> 8][ru][col & 255];
                        }
                        wd[k] = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
                    }
                }
            } else {
                const uint8_t *rowp = U_.in + (int64_t)(INTERIOR ? yin : clampi(yin, 0, h - 1)) * U_.in_pitch;
                if (!border && ((((uintptr_t)(rowp + xl)) & 15) == 0)) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(rowp + xl));
                    wd[0] = v.x; wd[1] = v.y; wd[2] = v.z; wd[3] = v.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        uint32_t b[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) b[e] = __ldg(rowp + clampi(xl + 4 * k + e, 0, w - 1));
                        wd[k] = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
                    }
                }
            }
            if (!INTERIOR && yin == h - 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) last[k] = wd[k];
            }

            // ---- Step 1, vertical: (1,2,1) on input rows -> a(yin-1), on a -> V(yin-2)
            const int z0 = u, z1 = (u + 2) % 3, z2 = (u + 1) % 3;       // slots of iterations i, i-1, i-2
            uint32_t v[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                rq[z0][k] = perm(wd[k], 0u, 0x4240u);
                rq[z0][k + 4] = perm(wd[k], 0u, 0x4341u);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                ra[z0][j] = rq[z2][j] + 2u * rq[z1][j] + rq[z0][j];        // <= 1020 per 16-bit lane
                v[j] = ra[z2][j] + 2u * ra[z1][j] + ra[z0][j];             // <= 4080
            }
            if (i < 4) continue;                  // vertical window still filling (warp-uniform)

            // ---- Step 1, horizontal binomial; V(x) pairs E = v[0..3], O = v[4..7]
            const uint32_t Rh = __shfl_down_sync(FULL, perm(v[0], v[4], 0x5410u), 1);   // (V16, V17)
            const uint32_t Lh = __shfl_up_sync(FULL, perm(v[3], v[7], 0x7632u), 1);     // (V-2, V-1)
            uint32_t SE[4], SO[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t A = k ? perm(v[k - 1], v[k], 0x5432u) : perm(Lh, v[0], 0x5410u);      // (V4k-2, V4k)
                const uint32_t B = k ? perm(v[k + 3], v[k + 4], 0x5432u) : perm(Lh, v[4], 0x5432u);  // (V4k-1, V4k+1)
                const uint32_t C = k < 3 ? perm(v[k], v[k + 1], 0x5432u) : perm(v[3], Rh, 0x5432u);  // (V4k+2, V4k+4)
                const uint32_t D = k < 3 ? perm(v[k + 4], v[k + 5], 0x5432u) : perm(v[7], Rh, 0x7632u); // (V4k+3, V4k+5)
                const uint32_t he = A + C + BIAS + 4u * (B + v[k + 4]) + 6u * v[k];   // (h4k, h4k+2)
                const uint32_t ho = B + D + BIAS + 4u * (v[k] + C) + 6u * v[k + 4];   // (h4k+1, h4k+3)
                // S = h >> 8 as fp16 1024 + S: the high byte of each lane under exponent byte 0x64
                SE[k] = perm(he, H1024, 0x7351u);
                SO[k] = perm(ho, H1024, 0x7351u);
            }
            // replicate border on S at the right image edge: S(w) = S(w - 1)
            if (wborder && border && e_last >= 0 && e_last < LPX - 1) {
#pragma unroll
                for (int p = 0; p < LPX - 1; ++p)
                    if (p == e_last) set_px(SE, SO, p + 1, get_px(SE, SO, p));
            }

            // ---- Step 2: Sobel. Dx = S(x+1) - S(x-1); T = S(x-1) + 2 S(x) + S(x+1) + 1024
            const uint32_t SLw = __shfl_up_sync(FULL, SO[3], 1);    // left lane's (S13, S15): hi = S(-1)
            const uint32_t SRw = __shfl_down_sync(FULL, SE[0], 1);  // right lane's (S0, S2): lo = S(16)
            uint32_t DX[8], TB[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t SB = k ? perm(SO[k - 1], SO[k], 0x5432u) : perm(SLw, SO[0], 0x5432u);   // (S4k-1, S4k+1)
                uint32_t SC = k < 3 ? perm(SE[k], SE[k + 1], 0x5432u) : perm(SE[3], SRw, 0x5432u); // (S4k+2, S4k+4)
                if (wborder) {
                    if (k == 0 && xl == 0) SB = perm(SE[0], SO[0], 0x5410u);               // S(-1) = S(0)
                    if (k == 3 && e_last == LPX - 1) SC = perm(SE[3], SO[3], 0x7632u);     // S(w) = S(w-1)
                }
                dx[z0][k] = hsub2(SO[k], SB);
                dx[z0][k + 4] = hsub2(SC, SE[k]);
                tb[z0][k] = hadd2(hadd2(hfma2(SE[k], HTWO, HM3072), SB), SO[k]);
                tb[z0][k + 4] = hadd2(hadd2(hfma2(SO[k], HTWO, HM3072), SE[k]), SC);
            }
            if (!INTERIOR && s == h) {            // S(h) = S(h - 1)
#pragma unroll
                for (int j = 0; j < 8; ++j) { dx[z0][j] = dx[z1][j]; tb[z0][j] = tb[z1][j]; }
            }
            uint32_t gx[8], gy[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                gx[j] = hadd2(hfma2(dx[z1][j], HTWO, dx[z2][j]), dx[z0][j]);   // Dx(r-1) + 2 Dx(r) + Dx(r+1)
                gy[j] = hsub2(tb[z0][j], tb[z2][j]);                           // T(r+1) - T(r-1)
            }
            if (!INTERIOR && s == 0) {            // S(-1) = S(0) for the next row's Sobel
#pragma unroll
                for (int j = 0; j < 8; ++j) { dx[z1][j] = dx[z0][j]; tb[z1][j] = tb[z0][j]; }
            }
            if (i < 6) continue;                  // Sobel rows start at Y0 - 1 (warp-uniform)

            // ---- outside the image the strengths are 0
            if (!INTERIOR) {
                if (r < 0 || r >= h) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) gx[j] = gy[j] = 0u;
                } else if (wborder && border) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int p0 = 4 * (j & 3) + (j >> 2), p1 = p0 + 2;   // pixels of pair j
                        const uint32_t keep = (xl + p0 >= 0 && p0 <= e_last ? 0x0000FFFFu : 0u) |
                                              (xl + p1 >= 0 && p1 <= e_last ? 0xFFFF0000u : 0u);
                        gx[j] &= keep;
                        gy[j] &= keep;
                    }
                }
            }
            uint8_t *grow = S.g[gsl];
            *reinterpret_cast<uint4 *>(grow + 0 * GHALF + lane * 16) = make_uint4(gx[0], gx[1], gx[2], gx[3]);
            *reinterpret_cast<uint4 *>(grow + 1 * GHALF + lane * 16) = make_uint4(gx[4], gx[5], gx[6], gx[7]);
            *reinterpret_cast<uint4 *>(grow + 2 * GHALF + lane * 16) = make_uint4(gy[0], gy[1], gy[2], gy[3]);
            *reinterpret_cast<uint4 *>(grow + 3 * GHALF + lane * 16) = make_uint4(gy[4], gy[5], gy[6], gy[7]);
            gsl = gsl == GRING - 1 ? 0 : gsl + 1;

            // ---- candidates: Gx^2 + Gy^2 - L' >= 0 in fp16 (sign bit clear)
            uint32_t acc = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t de = hfma2(gx[k], gx[k], hfma2(gy[k], gy[k], negL));
                const uint32_t dd = hfma2(gx[k + 4], gx[k + 4], hfma2(gy[k + 4], gy[k + 4], negL));
                const uint32_t wq = perm(de, dd, 0x7351u);   // sign bytes of pixels 4k, 4k+1, 4k+2, 4k+3
                if (k == 0) acc = wq;
                else {
                    const uint32_t sel = (0xFF00u >> k) & 0xFFu;
                    const uint32_t c = sel * 0x01010101u;    // bits 7 .. 8-k of each byte keep acc
                    acc = (acc & c) | ((wq >> k) & ~c);
                }
            }
            uint32_t m = ~acc & 0xF0F0F0F0u;
            const bool in_band = INTERIOR ? (i >= 7 && i < BAND + 7) : (i >= 7 && i < BAND + 7 && r < h);
            if (!in_band || !out_lane) m = 0u;
            if (u < U - 1) mk[u + 1] = m;
            else carry = m;
        }

        // ---- refill the stage this group consumed
        if (TMA) {
            __syncwarp();
            if (lane == 0 && g + STAGES < GROUPS && !failed) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue_chunk(g + STAGES);
            }
        }

        // ---- Step 3 + thresholds for the flagged pixels of rows R .. R+U-1 (R = Y0 + U g - 8)
        const int R = Y0 + U * g - 8;
        __syncwarp();
        uint32_t anyf = 0u;
#pragma unroll
        for (int rr = 0; rr < U; ++rr) anyf |= mk[rr];
        if (g >= 2 && __any_sync(FULL, anyf != 0u)) {
            // ring slot of row R: rows Y0-1+k sit in slot k mod GRING and gsl follows row R+U
            const int slotR = gsl == GRING - 1 ? 0 : gsl + 1;
            uint32_t pre[U];                      // flags of this lane in rows before rr, inclusive of rr
            uint32_t cnt = 0u;
#pragma unroll
            for (int rr = 0; rr < U; ++rr) {
                pre[rr] = (rr ? pre[rr - 1] : 0u) + __popc(mk[rr]);
                if (rr < U - 1) cnt |= pre[rr] << (8 * rr);
            }
            const uint32_t cl = pre[U - 1];
            uint32_t incl = cl;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(FULL, incl, d);
                if (lane >= d) incl += o;
            }
            const uint32_t n = __shfl_sync(FULL, incl, 31);
#pragma unroll 1
            for (uint32_t base = 0; base < n; base += 32) {
                // flagged pixel j of the warp (in lane, row, pixel order) goes to lane j - base;
                // its owner is the first lane whose inclusive count exceeds j
                const uint32_t j = base + lane;
                int own = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (__shfl_sync(FULL, incl, own + step - 1) <= j) own += step;
                const uint32_t o_excl = __shfl_sync(FULL, incl - cl, own);
                const uint32_t o_cnt = __shfl_sync(FULL, cnt, own);
                uint32_t om[U];
#pragma unroll
                for (int rr = 0; rr < U; ++rr) om[rr] = __shfl_sync(FULL, mk[rr], own);
                if (j < n) {
                    uint32_t k = j - o_excl, mw = om[0], kbase = 0u;
                    int rr = 0;
#pragma unroll
                    for (int q = 1; q < U; ++q) {
                        const uint32_t bq = (o_cnt >> (8 * (q - 1))) & 255u;
                        if (k >= bq) { rr = q; mw = om[q]; kbase = bq; }
                    }
                    const int col = own * LPX + flag_px(nth_flag(mw, k - kbase));
                    int sc = slotR + rr;
                    if (sc >= GRING) sc -= GRING;
                    const int su = sc == 0 ? GRING - 1 : sc - 1, sd = sc == GRING - 1 ? 0 : sc + 1;
                    suppress_pixel(S, col, S.g[sc], S.g[su], S.g[sd], (R + rr - Y0) % CROWS, lo2, hi2, err);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int rr = 0; rr < U - 1; ++rr) mk[rr] = 0u;
        mk[0] = carry;

        // ---- Step 4, tile-local: once the last row of a tile row is classified
        if (next_tile < Band<BAND>::TILES_Y && R + U - 1 >= Y0 + HT * next_tile + HT - 1) {
            finish_tile_row<BAND, MODE>(S, U_, O, next_tile, lane);
            ++next_tile;
        }
    }
}

// A unit away from every image border: input rows Y0 - 4 .. Y0 + ITERS - 5 and
// the columns of all 32 lanes (X0 - 16 .. X0 + 495) in the image.
template <int BAND>
__device__ __forceinline__ bool interior_unit(const Unit &U_)
{
    return U_.X0 >= LPX && U_.X0 + OUT_W + LPX <= U_.w && U_.Y0 >= 4 && U_.Y0 + Band<BAND>::ITERS - 4 <= U_.h;
}

// PATH: 0 = per unit (U.tma), 1 = TMA only, 2 = direct loads only. A kernel that
// holds one path only is compiled for that path alone (no register pressure
// from the other).
enum { PATH_EITHER = 0, PATH_TMA = 1, PATH_DIRECT = 2 };

// SPLIT: interior units take the stencil compiled without border checks. The
// batch kernel, whose units are mostly border units of small images, holds the
// general stencil alone.
template <int BAND, int MODE, int PATH, bool SPLIT>
__device__ __forceinline__ void run_unit(const CUtensorMap *tmap, const Unit &U_, IntThresholds t, const Out &O,
                                         uint32_t pbase, uint32_t *err, Smem &S, int lane)
{
    for (int k = lane; k < CROWS * TILES_X; k += THREADS) {
        (&S.cand[0][0])[k] = 0u;
        (&S.strong[0][0])[k] = 0u;
    }
    __syncwarp();
    if (PATH == PATH_TMA || (PATH == PATH_EITHER && U_.tma)) {
        // the previous unit's reads of the stage buffers are done before TMA reuses them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (PATH != PATH_DIRECT) {
            if (SPLIT && interior_unit<BAND>(U_))
                stencil_band<true, BAND, true, MODE>(tmap, U_, t, O, S, lane, pbase, err);
            else
                stencil_band<true, BAND, false, MODE>(tmap, U_, t, O, S, lane, pbase, err);
        }
    } else {
        if constexpr (PATH != PATH_TMA) {
            if (SPLIT && interior_unit<BAND>(U_))
                stencil_band<false, BAND, true, MODE>(tmap, U_, t, O, S, lane, pbase, err);
            else
                stencil_band<false, BAND, false, MODE>(tmap, U_, t, O, S, lane, pbase, err);
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void init_barriers(Smem &S, int lane)
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
__global__ void __launch_bounds__(THREADS, 12)
k1_fused_kernel(const __grid_constant__ CUtensorMap tmap, const uint8_t *__restrict__ in, int in_pitch,
                int w, int h, IntThresholds t, uint8_t *__restrict__ out, int out_pitch,
                HystScratch hs, HystImage img, uint32_t *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int lane = threadIdx.x;
    init_barriers(S, lane);
    Unit U_;
    U_.in = in;
    U_.in_pitch = in_pitch;
    U_.w = w;
    U_.h = h;
    U_.sx = blockIdx.x;
    // the bottom band row (border units, the slower stencil) starts right after
    // the top one instead of in the last wave: bands 0, nb - 1, 1, 2, ..., nb - 2
    const int nb = (int)gridDim.y, by = (int)blockIdx.y;
    U_.sy = by == 0 || nb < 3 ? by : (by == 1 ? nb - 1 : by - 1);
    U_.X0 = U_.sx * OUT_W;
    U_.Y0 = U_.sy * BAND;
    U_.tma = PATH == PATH_TMA;
    Out O;
    O.map = out;
    O.pitch = out_pitch;
    O.hs = hs;
    O.img = img;
    run_unit<BAND, MODE, PATH, true>(&tmap, U_, t, O, 0u, err, S, lane);
}

// One (image, strip, band) unit of a batch.
template <int BAND, int PATH>
__device__ __forceinline__ void batch_unit(const BatchImage *__restrict__ imgs, const CUtensorMap *__restrict__ tmaps,
                                           int nimg, uint32_t unit, IntThresholds t, const HystScratch &hs,
                                           uint32_t pbase, Smem &S, int lane)
{
    int lo = 0, hi = nimg - 1;                     // last image whose units start at or before unit
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].unit_base <= unit) lo = mid;
        else hi = mid - 1;
    }
    const BatchImage &B = imgs[lo];
    const uint32_t local = unit - B.unit_base;
    Unit U_;
    U_.in = B.in;
    U_.in_pitch = B.in_pitch;
    U_.w = B.img.w;
    U_.h = B.img.h;
    U_.sx = (int)(local % (uint32_t)B.nsx);
    U_.sy = (int)(local / (uint32_t)B.nsx);
    U_.X0 = U_.sx * OUT_W;
    U_.Y0 = U_.sy * BAND;
    U_.tma = PATH == PATH_TMA || B.tma != 0;
    Out O;
    O.img = B.img;
    O.map = O.img.map;
    O.pitch = O.img.pitch;
    O.hs = hs;
    if (U_.tma && lane == 0) {
        // the descriptor was rewritten in global memory since the TMA unit may
        // last have cached one at this address: order that write before its use
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&tmaps[lo]) : "memory");
    }
    __syncwarp();
    run_unit<BAND, MODE_EDGES, PATH, false>(&tmaps[lo], U_, t, O, pbase, &hs.state->error, S, lane);
}

// A batch. PERSIST: a persistent grid pops units from a counter; otherwise the
// grid has one CTA per unit (set per launch) and the hardware schedules them.
// PATH_TMA when every input is TMA-readable, else PATH_EITHER (chosen per image).
template <int BAND, int PATH, bool PERSIST>
__global__ void __launch_bounds__(THREADS, 12)
k1_fused_batch_kernel(const BatchImage *__restrict__ imgs, const CUtensorMap *__restrict__ tmaps,
                      BatchHeader *hdr, IntThresholds t, HystScratch hs)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int lane = threadIdx.x;
    const uint32_t total = hdr->total_units;
    const int nimg = (int)hdr->nimg;
    if constexpr (!PERSIST) {
        if (blockIdx.x >= total) return;
        init_barriers(S, lane);
        batch_unit<BAND, PATH>(imgs, tmaps, nimg, blockIdx.x, t, hs, 0u, S, lane);
    } else {
        init_barriers(S, lane);
        // each stage completes GROUPS / STAGES phases per TMA unit: track the parity
        uint32_t pbase = 0u;
        for (;;) {
            uint32_t unit = 0;
            if (lane == 0) unit = atomicAdd(&hdr->next_unit, 1u);
            unit = __shfl_sync(FULL, unit, 0);
            if (unit >= total) break;
            batch_unit<BAND, PATH>(imgs, tmaps, nimg, unit, t, hs, pbase, S, lane);
            // a direct-load unit leaves the barriers untouched; the image decides
            int lo = 0, hi = nimg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (imgs[mid].unit_base <= unit) lo = mid;
                else hi = mid - 1;
            }
            if (PATH == PATH_TMA || imgs[lo].tma != 0) pbase ^= (uint32_t)((Band<BAND>::GROUPS / STAGES) & 1);
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
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k1_fused_kernel<BAND, MODE, PATH_DIRECT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((w + OUT_W - 1) / OUT_W, (h + BAND - 1) / BAND);
    if (tma)
        k1_fused_kernel<BAND, MODE, PATH_TMA><<<grid, THREADS, sizeof(Smem), s>>>(
            tmap, in, in_pitch, w, h, t, out, out_pitch, hs, img, err);
    else
        k1_fused_kernel<BAND, MODE, PATH_DIRECT><<<grid, THREADS, sizeof(Smem), s>>>(
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
    case 32: return launch_single<32, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    case 160: return launch_single<160, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    case 256: return launch_single<256, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    default: return launch_single<64, MODE>(tmap, tma, in, in_pitch, w, h, t, out, out_pitch, hs, img, err, s);
    }
}

}  // namespace

bool k1_band_supported(int band) { return band == 32 || band == 64 || band == 160 || band == 256; }

int k1_band_rows(int band)
{
    switch (band) {
    case 32: return Band<32>::ITERS;
    case 160: return Band<160>::ITERS;
    case 256: return Band<256>::ITERS;
    default: return Band<64>::ITERS;
    }
}

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
    cudaError_t e = launch_any<MODE_EDGES>(band, in, in_pitch, w, h, t, img.map, img.pitch, hs, img,
                                           &hs.state->error, s);
    if (e == cudaSuccess) e = launch_hyst_fill_single(hs, img, s);
    return e;
}

// Kernel node parameters of the batch kernel; grid: CTAs (persistent) or units.
template <int BAND, int PATH, bool PERSIST>
cudaError_t batch_node_params(const BatchImage *const &imgs, const CUtensorMap *const &tmaps, BatchHeader *const &hdr,
                              const IntThresholds &t, const HystScratch &hs, unsigned grid, void **args,
                              cudaKernelNodeParams *kp)
{
    cudaError_t e = cudaFuncSetAttribute(k1_fused_batch_kernel<BAND, PATH, PERSIST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
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
    kp->sharedMemBytes = sizeof(Smem);
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
    case 32: return batch_params_band<32>(tma_only, persist, imgs, tmaps, hdr, t, hs, grid, args, kp);
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
