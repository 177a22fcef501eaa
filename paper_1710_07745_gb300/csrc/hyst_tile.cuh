// hyst_tile.cuh -- per-tile pieces of the hysteresis (Step 4 of the paper's
// Sec. 2.2.1) shared by the stand-alone local fill and the fused stencil:
// 32x32 tiles as 32-bit row masks in one warp (lane = row).
#pragma once

#include "canny_internal.cuh"

namespace canny {
namespace tile {

constexpr unsigned FULL = 0xffffffffu;
// Bits of c that lie in a run (of consecutive set bits) containing a bit of s;
// s must be a subset of c. Upward: adding s to c carries from the lowest seed of
// each run past its top, clearing exactly the bits from that seed up; downward:
// the same on the bit-reversed words.
__device__ __forceinline__ uint32_t fill_runs(uint32_t s, uint32_t c)
{
    uint32_t up = (c & ~(c + s)) | s;
    uint32_t rs = __brev(s), rc = __brev(c);
    uint32_t dn = __brev((rc & ~(rc + rs)) | rs);
    return up | dn;
}

// fill_runs with the bit reversal of c computed once by the caller.
__device__ __forceinline__ uint32_t fill_runs_r(uint32_t s, uint32_t c, uint32_t rc)
{
    uint32_t up = (c & ~(c + s)) | s;
    uint32_t rs = __brev(s);
    uint32_t dn = __brev((rc & ~(rc + rs)) | rs);
    return up | dn;
}

// A row mask and its left and right neighbours.
__device__ __forceinline__ uint32_t dilate(uint32_t x) { return x | (x << 1) | (x >> 1); }

// Grow e (subset of c) through 8-connected pixels of c inside the tile until
// stable (lane = row). A round pulls the masks of the four rows above and the
// four below and grows them in order towards the lane's own row (each row's
// runs filled, then the next row seeded from its dilation), so a chain climbs
// up to four rows per round instead of one. Every round that changes something
// adds at least one pixel, so at most 1024 + 1 rounds run.
__device__ __forceinline__ uint32_t flood_tile(uint32_t e, uint32_t c, int lane)
{
    const uint32_t rc = __brev(c);
    uint32_t ca[4], cb[4], rca[4], rcb[4];     // c of rows lane-1-k and lane+1+k (0 outside)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        ca[k] = __shfl_up_sync(FULL, c, k + 1);
        cb[k] = __shfl_down_sync(FULL, c, k + 1);
        if (lane < k + 1) ca[k] = 0u;
        if (lane + k + 1 > HT - 1) cb[k] = 0u;
        rca[k] = __brev(ca[k]);
        rcb[k] = __brev(cb[k]);
    }
    e = fill_runs_r(e, c, rc);
    for (int it = 0; it < HT * HT + 2; ++it) {
        uint32_t a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = __shfl_up_sync(FULL, e, k + 1) & ca[k];
            b[k] = __shfl_down_sync(FULL, e, k + 1) & cb[k];
        }
        uint32_t x = a[3], y = b[3];
#pragma unroll
        for (int k = 2; k >= 0; --k) {
            x = fill_runs_r(a[k] | (ca[k] & dilate(x)), ca[k], rca[k]);
            y = fill_runs_r(b[k] | (cb[k] & dilate(y)), cb[k], rcb[k]);
        }
        const uint32_t ne = fill_runs_r(e | (c & (dilate(x) | dilate(y))), c, rc);
        const bool changed = __any_sync(FULL, ne != e);
        e = ne;
        if (!changed) break;
    }
    return e;
}

// Four tiles per warp: lane 8 t + s holds rows 4 s .. 4 s + 3 of tile t, as
// e[0..3] (subsets of c[0..3]). Grows every tile's e through 8-connected pixels
// of its c until no tile changes. A round fills each row's runs while sweeping
// the lane's four rows down and back up, then passes the outer rows' neighbours
// to the lanes above and below in the same tile, so a chain climbs several rows
// per round. Every round that changes something adds a pixel, so at most
// 4 x 1024 + 1 rounds run.
__device__ __forceinline__ void flood4(uint32_t (&e)[4], const uint32_t (&c)[4], int sl)
{
    uint32_t rc[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) rc[r] = __brev(c[r]);
    for (int it = 0; it < 4 * HT * HT + 2; ++it) {
        const uint32_t o0 = e[0], o1 = e[1], o2 = e[2], o3 = e[3];
        e[0] = fill_runs_r(e[0], c[0], rc[0]);
#pragma unroll
        for (int r = 1; r < 4; ++r) e[r] = fill_runs_r(e[r] | (c[r] & dilate(e[r - 1])), c[r], rc[r]);
#pragma unroll
        for (int r = 2; r >= 0; --r) e[r] = fill_runs_r(e[r] | (c[r] & dilate(e[r + 1])), c[r], rc[r]);
        uint32_t a = __shfl_up_sync(FULL, dilate(e[3]), 1, 8);
        uint32_t b = __shfl_down_sync(FULL, dilate(e[0]), 1, 8);
        if (sl == 0) a = 0u;
        if (sl == 7) b = 0u;
        e[0] = fill_runs_r(e[0] | (c[0] & a), c[0], rc[0]);
        e[3] = fill_runs_r(e[3] | (c[3] & b), c[3], rc[3]);
        if (!__any_sync(FULL, ((e[0] ^ o0) | (e[1] ^ o1) | (e[2] ^ o2) | (e[3] ^ o3)) != 0u)) break;
    }
}

// 4-bit mask of the nonzero bytes of w (bit k = byte k).
__device__ __forceinline__ uint32_t nz_nibble(uint32_t w)
{
    uint32_t m = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
    return ((m >> 7) * 0x10204080u) >> 28;
}

// 4 bytes 0xFF/0x00 from the low 4 bits of t.
__device__ __forceinline__ uint32_t nibble_bytes(uint32_t t)
{
    return (((t & 0xFu) * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// Row `lane` of tile (tx, ty): cand = class >= 1, strong = class >= 2.
__device__ __forceinline__ void load_row(const HystImage &im, int tx, int ty, int lane,
                                         uint32_t &cand, uint32_t &strong)
{
    cand = strong = 0;
    int y = ty * HT + lane, x0 = tx * HT;
    if (y >= im.h) return;
    const uint8_t *row = im.map + (int64_t)y * im.pitch + x0;
    int n = min(HT, im.w - x0);
    if (n == HT && (((uintptr_t)row) & 15) == 0) {
        uint4 a = reinterpret_cast<const uint4 *>(row)[0];
        uint4 b = reinterpret_cast<const uint4 *>(row)[1];
        uint32_t wd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cand |= nz_nibble(wd[k]) << (4 * k);
            strong |= nz_nibble(wd[k] & 0xFEFEFEFEu) << (4 * k);
        }
    } else {
        for (int i = 0; i < n; ++i) {
            uint8_t v = row[i];
            if (v) cand |= 1u << i;
            if (v >= 2) strong |= 1u << i;
        }
    }
}

// Store 32 bytes (little-endian words wd[0..7]) at p, any alignment, with the
// widest stores the alignment allows: two 16-byte stores when 16-byte aligned,
// 8- or 4-byte words when 8- or 4-byte aligned, otherwise seven 4-byte words
// funnel-shifted into place between a head and a tail of one byte and/or one
// 16-bit store (at most 11 stores instead of 32).
__device__ __forceinline__ void store32(uint8_t *p, const uint32_t (&wd)[8])
{
    const uintptr_t a = (uintptr_t)p;
    const int r = (int)(a & 3);
    if ((a & 15) == 0) {
        reinterpret_cast<uint4 *>(p)[0] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        reinterpret_cast<uint4 *>(p)[1] = make_uint4(wd[4], wd[5], wd[6], wd[7]);
    } else if ((a & 7) == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) reinterpret_cast<uint2 *>(p)[k] = make_uint2(wd[2 * k], wd[2 * k + 1]);
    } else if (r == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) reinterpret_cast<uint32_t *>(p)[k] = wd[k];
    } else {
        // aligned word k of the destination (at p - r + 4k) holds data bytes 4k - r .. 4k - r + 3
        uint32_t *base = reinterpret_cast<uint32_t *>(p - r);
        const uint32_t sh = 8u * (uint32_t)(4 - r);
#pragma unroll
        for (int k = 1; k < 8; ++k) base[k] = __funnelshift_r(wd[k - 1], wd[k], sh);
        // head: data bytes 0 .. 3 - r; tail: data bytes 32 - r .. 31
        if (r & 1) p[0] = (uint8_t)wd[0];
        if (r != 3) *reinterpret_cast<uint16_t *>(p + (r & 1)) = (uint16_t)(wd[0] >> (8 * (r & 1)));
        if (r != 1) *reinterpret_cast<uint16_t *>(p + 32 - r) = (uint16_t)(wd[7] >> sh);
        if (r & 1) p[31] = (uint8_t)(wd[7] >> 24);
    }
}

// Write row `lane` of the tile as 255 where e is set, 0 elsewhere.
__device__ __forceinline__ void store_row(const HystImage &im, int tx, int ty, int lane, uint32_t e)
{
    int y = ty * HT + lane, x0 = tx * HT;
    if (y >= im.h) return;
    uint8_t *row = im.map + (int64_t)y * im.pitch + x0;
    int n = min(HT, im.w - x0);
    if (n < HT) {
        for (int i = 0; i < n; ++i) row[i] = ((e >> i) & 1) ? 255 : 0;
        return;
    }
    uint32_t wd[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) wd[k] = nibble_bytes(e >> (4 * k));
    store32(row, wd);
}

// Write image row y of tile column tx as 255 where e is set, 0 elsewhere.
__device__ __forceinline__ void store_tile_row(const HystImage &im, int tx, int y, uint32_t e)
{
    const int x0 = tx * HT;
    if (y >= im.h) return;
    uint8_t *row = im.map + (int64_t)y * im.pitch + x0;
    const int n = min(HT, im.w - x0);
    if (n < HT) {
        for (int i = 0; i < n; ++i) row[i] = ((e >> i) & 1) ? 255 : 0;
        return;
    }
    uint32_t wd[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) wd[k] = nibble_bytes(e >> (4 * k));
    store32(row, wd);
}

// Finish four tiles at once (lane 8 tt + sl holds rows 4 sl .. 4 sl + 3 of its
// tile): grow the edges e (the strong pixels) through the candidates c, write the
// tile's edge rows as 255/0, its border masks, pending bitmap and queue stamp.
// valid: the lane's tile exists (tile index tid at (tx, ty) of image im); the
// other lanes pass c = e = 0.
// Returns, on the tile's first lane, bit 0: queue the tile for pass 0, bit 1: it
// has pending pixels (the caller counts them and fills the worklist).
__device__ __forceinline__ uint32_t finish4(const HystScratch &hs, const HystImage &im, int tx, int ty, uint32_t tid,
                                            bool valid, const uint32_t (&c)[4], uint32_t (&e)[4], int lane)
{
    const int tt = lane >> 3, sl = lane & 7;
    if (__any_sync(FULL, ((c[0] ^ e[0]) | (c[1] ^ e[1]) | (c[2] ^ e[2]) | (c[3] ^ e[3])) != 0u)) flood4(e, c, sl);
    uint32_t pend[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) pend[r] = c[r] & ~e[r];
    // border columns: each lane's four bits, gathered over the tile's eight lanes
    uint32_t el = 0u, er = 0u, pl = 0u, pr = 0u;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        el |= (e[r] & 1u) << r;
        er |= (e[r] >> 31) << r;
        pl |= (pend[r] & 1u) << r;
        pr |= (pend[r] >> 31) << r;
    }
    el <<= 4 * sl;
    er <<= 4 * sl;
    pl <<= 4 * sl;
    pr <<= 4 * sl;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        el |= __shfl_xor_sync(FULL, el, d);
        er |= __shfl_xor_sync(FULL, er, d);
        pl |= __shfl_xor_sync(FULL, pl, d);
        pr |= __shfl_xor_sync(FULL, pr, d);
    }
    TileMasks m;
    m.edge_top = __shfl_sync(FULL, e[0], lane & ~7);
    m.edge_bottom = __shfl_sync(FULL, e[3], lane | 7);
    m.pend_top = __shfl_sync(FULL, pend[0], lane & ~7);
    m.pend_bottom = __shfl_sync(FULL, pend[3], lane | 7);
    m.edge_left = el;
    m.edge_right = er;
    m.pend_left = pl;
    m.pend_right = pr;
    const uint32_t pbal = __ballot_sync(FULL, (pend[0] | pend[1] | pend[2] | pend[3]) != 0u);
    const bool any_pend = ((pbal >> (8 * tt)) & 0xFFu) != 0u;
    if (!valid) return 0u;
    const int y0 = ty * HT + 4 * sl;
    const bool fast = ((((uintptr_t)im.map) | (uintptr_t)im.pitch) & 15) == 0 && (tx + 1) * HT <= im.w &&
                      (ty + 1) * HT <= im.h;
    if (fast) {
        // whole tile in 16-byte aligned rows: two 16-byte stores a row
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            uint4 *p = reinterpret_cast<uint4 *>(im.map + (int64_t)(y0 + r) * im.pitch + tx * HT);
            p[0] = make_uint4(nibble_bytes(e[r]), nibble_bytes(e[r] >> 4), nibble_bytes(e[r] >> 8),
                              nibble_bytes(e[r] >> 12));
            p[1] = make_uint4(nibble_bytes(e[r] >> 16), nibble_bytes(e[r] >> 20), nibble_bytes(e[r] >> 24),
                              nibble_bytes(e[r] >> 28));
        }
    } else {
#pragma unroll 1
        for (int r = 0; r < 4; ++r) store_tile_row(im, tx, y0 + r, e[r]);
    }
    if (!CANNY_CHECK(tid < hs.max_tiles, &hs.state->error)) return 0u;
    if (any_pend)
        *reinterpret_cast<uint4 *>(&hs.pend_bits[(size_t)tid * HT + 4 * sl]) = make_uint4(pend[0], pend[1], pend[2], pend[3]);
    if (sl != 0) return 0u;
    hs.masks[tid] = m;
    // pending pixels on the border may be reached from a neighbour: queue for
    // pass 0 (1 = queued for pass 0, 0 = not queued; every tile writes its stamp)
    const bool queue = (m.pend_top | m.pend_bottom | m.pend_left | m.pend_right) != 0u;
    hs.stamp[tid] = queue ? 1u : 0u;
    return (queue ? 1u : 0u) | (any_pend ? 2u : 0u);
}

__device__ __forceinline__ int find_image(const HystImage *imgs, int nimg, uint32_t t)
{
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (imgs[mid].tile_base <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void push(const HystScratch &hs, uint32_t list, uint32_t tile, uint32_t stamp)
{
    if (atomicMax(&hs.stamp[tile], stamp) < stamp) {
        uint32_t idx = atomicAdd(&hs.state->list_count[list], 1u);
        if (CANNY_CHECK(idx < hs.max_tiles && tile < hs.max_tiles, &hs.state->error))
            hs.lists[(size_t)list * hs.max_tiles + idx] = tile;
    }
}


// Border masks, pending bitmap and first-worklist entry of tile t once its
// final edge set e and candidate set cand are known (all lanes call).
__device__ __forceinline__ void finish_tile(const HystScratch &hs, uint32_t t, uint32_t e, uint32_t cand,
                                            int lane)
{
    const uint32_t pend = cand & ~e;
    TileMasks m;
    m.edge_top = __shfl_sync(FULL, e, 0);
    m.edge_bottom = __shfl_sync(FULL, e, HT - 1);
    m.edge_left = __ballot_sync(FULL, e & 1u);
    m.edge_right = __ballot_sync(FULL, e >> 31);
    m.pend_top = __shfl_sync(FULL, pend, 0);
    m.pend_bottom = __shfl_sync(FULL, pend, HT - 1);
    m.pend_left = __ballot_sync(FULL, pend & 1u);
    m.pend_right = __ballot_sync(FULL, pend >> 31);
    const bool any_pend = __any_sync(FULL, pend != 0);
    if (!CANNY_CHECK(t < hs.max_tiles, &hs.state->error)) return;
    if (any_pend) hs.pend_bits[(size_t)t * HT + lane] = pend;
    if (lane == 0) {
        hs.masks[t] = m;
        if (any_pend) atomicAdd(&hs.state->pending_tiles, 1u);
        // pending pixels on the border may be reached from a neighbour: queue for pass 0
        // every tile of a run writes its own stamp here, so no clearing pass is needed:
        // 1 = queued for pass 0, 0 = not queued
        const bool queue = (m.pend_top | m.pend_bottom | m.pend_left | m.pend_right) != 0;
        hs.stamp[t] = queue ? 1u : 0u;
        if (queue) {
            const uint32_t i = atomicAdd(&hs.state->list_count[0], 1u);
            if (CANNY_CHECK(i < hs.max_tiles, &hs.state->error)) hs.lists[i] = t;
        }
    }
}

}  // namespace tile
}  // namespace canny
