// hysteresis.cu -- Step 4 of the paper's Sec. 2.2.1: a weak pixel (between the
// thresholds) is an edge only if it is connected to a strong one. Read as
// 8-connectivity through weak/strong pixels.
//
// Two stages, both on 32x32 tiles held as 32-bit row masks in one warp
// (lane = row):
//   local fill   each tile grows its strong pixels through its own weak pixels
//                until stable, writes 255/0 into the map, and records which weak
//                pixels are still unresolved ("pending") and which border pixels
//                are edges or pending;
//   global pass  a tile on the worklist takes the edges on its neighbours'
//                borders as seeds for its pending border pixels and grows them
//                (the lanes of a warp first check a chunk of entries for seeds
//                at once). A neighbour whose facing border gained edges next
//                to its pending pixels is followed at once by the same warp;
//                in the cooperative launch (every CTA resident) further seeded
//                entries and branches go to an in-pass queue that idle warps
//                drain, in one launch per pass to the warp's own stack; what
//                the budget cannot take is listed for the next pass. Passes
//                repeat until the
//                worklist is empty, decided by the last CTA of each pass: for a
//                single image all passes run in one cooperative launch (a
//                bounded grid barrier between them); inside the batch and
//                frame graphs a CUDA-graph while-node drives the loop.
// Pending pixels live only in a compact bitmap, so the map never holds a value
// other than 0/255 and no clean-up sweep is needed.
#include <algorithm>

#include "hyst_tile.cuh"

namespace canny {

namespace {

constexpr int WARPS = 8;             // tiles per CTA in the local fill and the global pass
constexpr int THREADS = WARPS * 32;
using namespace tile;

// ---------------------------------------------------------------- local fill
template <bool SINGLE>
__global__ void __launch_bounds__(THREADS)
hyst_local_kernel(HystScratch hs, HystImage single, uint32_t ntiles, uint32_t nimg)
{
    const int lane = threadIdx.x & 31;
    const uint32_t t = (blockIdx.x * THREADS + threadIdx.x) >> 5;
    if (SINGLE && blockIdx.x == 0 && threadIdx.x == 0) hs.imgs[0] = single;
    if (t >= ntiles) return;
    HystImage im = SINGLE ? single : hs.imgs[find_image(hs.imgs, (int)nimg, t)];
    const uint32_t local = t - im.tile_base;
    const int tx = (int)(local % (uint32_t)im.ntx), ty = (int)(local / (uint32_t)im.ntx);

    uint32_t cand, strong;
    load_row(im, tx, ty, lane, cand, strong);
    const uint32_t e = flood_tile(strong, cand, lane);
    store_row(im, tx, ty, lane, e);
    finish_tile(hs, t, e, cand, lane);
}

// ---------------------------------------------------------------- global pass
// Neighbour directions of a tile, as bits of the "affected" mask.
enum { NB_U, NB_UL, NB_UR, NB_D, NB_DL, NB_DR, NB_L, NB_R };

// Tiles a chain may be followed into within a pass before the rest is listed
// for the next pass (the default of the chase budget).
constexpr int CHASE_BUDGET = 16;
// The one-launch-per-pass kernel's default budget per worklist entry, and the
// depth of its per-warp chase stack.
constexpr int STACK_BUDGET = 64;
constexpr int CHASE_STACK = 32;
// The union-find stage follows the first pass only when that pass's worklist
// held at most this many tiles: its cost grows with the tiles it labels, a
// pass's with the length of the chains it follows, so images with many short
// chains (a large list) keep to passes.
constexpr uint32_t UF_MAX_ENTRIES = 32768;

// Border masks as other warps last wrote them: loads that bypass L1, since
// tiles are revisited within one pass and L1 is not coherent across SMs.
__device__ __forceinline__ TileMasks masks_cg(const TileMasks *m)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(m);
    const uint4 a = __ldcg(p), b = __ldcg(p + 1);
    TileMasks r;
    r.edge_top = a.x; r.edge_bottom = a.y; r.edge_left = a.z; r.edge_right = a.w;
    r.pend_top = b.x; r.pend_bottom = b.y; r.pend_left = b.z; r.pend_right = b.w;
    return r;
}

__device__ __forceinline__ uint32_t edge_bottom_cg(const TileMasks *m) { return __ldcg(&m->edge_bottom); }
__device__ __forceinline__ uint32_t edge_top_cg(const TileMasks *m) { return __ldcg(&m->edge_top); }
__device__ __forceinline__ uint32_t edge_left_cg(const TileMasks *m) { return __ldcg(&m->edge_left); }
__device__ __forceinline__ uint32_t edge_right_cg(const TileMasks *m) { return __ldcg(&m->edge_right); }

// Write 255 at the pixels of e (row `lane` of tile (tx, ty); whole warp). The
// other bytes of the rows may be edges already, so only e's bytes are stored:
// lane by lane (as many rounds as the fullest row has bits) or row by row (one
// coalesced store per row that has any), whichever takes fewer rounds.
__device__ __forceinline__ void store_new_edges(const HystImage &im, int tx, int ty, int lane, uint32_t e)
{
    const uint32_t rows = __ballot_sync(FULL, e != 0u);
    if (!rows) return;
    const int most = (int)__reduce_max_sync(FULL, (unsigned)__popc(e));
    if (__popc(rows) < most) {
        uint8_t *col = im.map + (int64_t)ty * HT * im.pitch + tx * HT + lane;
        for (uint32_t m = rows; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            if ((__shfl_sync(FULL, e, r) >> lane) & 1u) col[(int64_t)r * im.pitch] = 255;
        }
    } else {
        uint8_t *row = im.map + (int64_t)(ty * HT + lane) * im.pitch + tx * HT;
        for (uint32_t bits = e; bits; bits &= bits - 1) row[__ffs(bits) - 1] = 255;
    }
}

// Neighbour of tile t in direction d (NB_*) for an image ntx tiles wide:
// t + dy * ntx + dx, with dx + 1 and dy + 1 packed two bits per direction.
__device__ __forceinline__ uint32_t neighbour(uint32_t t, int d, uint32_t ntx)
{
    const int dx = (int)((0x8861u >> (2 * d)) & 3u) - 1;    // 0, -1, 1, 0, -1, 1, -1, 1
    const int dy = (int)((0x5A80u >> (2 * d)) & 3u) - 1;    // -1, -1, -1, 1, 1, 1, 0, 0
    return (uint32_t)((int64_t)t + (int64_t)dy * ntx + dx);
}

// Where tile t sits, and which of its pending border pixels touch an edge pixel
// of a neighbouring tile (the seeds of its growth). Lane-independent: a warp
// calls it for one tile, or each lane for its own.
struct TileSeeds {
    HystImage im;
    int tx, ty;
    uint32_t top, bot, left, right;
};

__device__ __forceinline__ bool find_seeds(const HystScratch &hs, uint32_t t, int nimg, TileSeeds &sd)
{
    sd.im = hs.imgs[find_image(hs.imgs, nimg, t)];      // read-only during the pass: cached
    const HystImage &im = sd.im;
    const uint32_t local = t - im.tile_base;
    const int tx = (int)(local % (uint32_t)im.ntx), ty = (int)(local / (uint32_t)im.ntx);
    sd.tx = tx;
    sd.ty = ty;
    const bool hasL = tx > 0, hasR = tx < im.ntx - 1, hasU = ty > 0, hasD = ty < im.nty - 1;
    const uint32_t ntx = (uint32_t)im.ntx;
    const TileMasks *M = hs.masks;
    // every word this test may need, loaded at once (one round trip to L2)
    const TileMasks mu = masks_cg(&M[t]);
    const uint32_t eu = hasU ? edge_bottom_cg(&M[t - ntx]) : 0u;
    const uint32_t eul = hasU && hasL ? edge_bottom_cg(&M[t - ntx - 1]) : 0u;
    const uint32_t eur = hasU && hasR ? edge_bottom_cg(&M[t - ntx + 1]) : 0u;
    const uint32_t ed = hasD ? edge_top_cg(&M[t + ntx]) : 0u;
    const uint32_t edl = hasD && hasL ? edge_top_cg(&M[t + ntx - 1]) : 0u;
    const uint32_t edr = hasD && hasR ? edge_top_cg(&M[t + ntx + 1]) : 0u;
    const uint32_t el = hasL ? edge_right_cg(&M[t - 1]) : 0u;
    const uint32_t er = hasR ? edge_left_cg(&M[t + 1]) : 0u;
    // pending border pixels next to an edge pixel of a neighbouring tile
    const uint32_t ring_top = eu | (eu << 1) | (eu >> 1) | (eul >> 31) | ((eur & 1u) << 31);
    const uint32_t ring_bot = ed | (ed << 1) | (ed >> 1) | (edl >> 31) | ((edr & 1u) << 31);
    sd.top = ring_top & mu.pend_top;
    sd.bot = ring_bot & mu.pend_bottom;
    sd.left = (el | (el << 1) | (el >> 1)) & mu.pend_left;
    sd.right = (er | (er << 1) | (er >> 1)) & mu.pend_right;
    return (sd.top | sd.bot | sd.left | sd.right) != 0;
}

// The pending border words of t's neighbours that face t (the pixels an edge on
// t's border would seed), as lane 0 read them at the start of a chase step.
struct Facing {
    uint32_t u, ul, ur, d, dl, dr, l, r;
};

// find_seeds for the tile a warp chases into, with every mask word read by lane
// 0 alone: the same thread made this warp's earlier updates of those words (its
// atomics in grow_tile), so it reads them back without a fence. Lane 0 also
// reads the neighbours' facing pending words for grow_tile, in the same round
// trip; the seeds are broadcast to every lane.
__device__ __forceinline__ bool chase_seeds(const HystScratch &hs, uint32_t t, int nimg, TileSeeds &sd, int lane,
                                            Facing &fp)
{
    sd.im = hs.imgs[find_image(hs.imgs, nimg, t)];
    const HystImage &im = sd.im;
    const uint32_t local = t - im.tile_base;
    const int tx = (int)(local % (uint32_t)im.ntx), ty = (int)(local / (uint32_t)im.ntx);
    sd.tx = tx;
    sd.ty = ty;
    uint32_t top = 0, bot = 0, left = 0, right = 0;
    fp = Facing{0, 0, 0, 0, 0, 0, 0, 0};
    if (lane == 0) {
        const bool hasL = tx > 0, hasR = tx < im.ntx - 1, hasU = ty > 0, hasD = ty < im.nty - 1;
        const uint32_t ntx = (uint32_t)im.ntx;
        const TileMasks *M = hs.masks;
        const TileMasks mu = masks_cg(&M[t]);
        uint32_t eu = 0, eul = 0, eur = 0, ed = 0, edl = 0, edr = 0, el = 0, er = 0;
        if (hasU) { eu = __ldcg(&M[t - ntx].edge_bottom); fp.u = __ldcg(&M[t - ntx].pend_bottom); }
        if (hasU && hasL) { eul = __ldcg(&M[t - ntx - 1].edge_bottom); fp.ul = __ldcg(&M[t - ntx - 1].pend_bottom); }
        if (hasU && hasR) { eur = __ldcg(&M[t - ntx + 1].edge_bottom); fp.ur = __ldcg(&M[t - ntx + 1].pend_bottom); }
        if (hasD) { ed = __ldcg(&M[t + ntx].edge_top); fp.d = __ldcg(&M[t + ntx].pend_top); }
        if (hasD && hasL) { edl = __ldcg(&M[t + ntx - 1].edge_top); fp.dl = __ldcg(&M[t + ntx - 1].pend_top); }
        if (hasD && hasR) { edr = __ldcg(&M[t + ntx + 1].edge_top); fp.dr = __ldcg(&M[t + ntx + 1].pend_top); }
        if (hasL) { el = __ldcg(&M[t - 1].edge_right); fp.l = __ldcg(&M[t - 1].pend_right); }
        if (hasR) { er = __ldcg(&M[t + 1].edge_left); fp.r = __ldcg(&M[t + 1].pend_left); }
        const uint32_t ring_top = eu | (eu << 1) | (eu >> 1) | (eul >> 31) | ((eur & 1u) << 31);
        const uint32_t ring_bot = ed | (ed << 1) | (ed >> 1) | (edl >> 31) | ((edr & 1u) << 31);
        top = ring_top & mu.pend_top;
        bot = ring_bot & mu.pend_bottom;
        left = (el | (el << 1) | (el >> 1)) & mu.pend_left;
        right = (er | (er << 1) | (er >> 1)) & mu.pend_right;
    }
    sd.top = __shfl_sync(FULL, top, 0);
    sd.bot = __shfl_sync(FULL, bot, 0);
    sd.left = __shfl_sync(FULL, left, 0);
    sd.right = __shfl_sync(FULL, right, 0);
    return (sd.top | sd.bot | sd.left | sd.right) != 0;
}

// Tile t grows its seeds through its pending pixels (whole warp, lane = row).
// Returns (in every lane) the mask of neighbours (NB_* bits) whose facing
// border has pending pixels next to an edge this call added, judged on the
// facing words lane 0 read in chase_seeds (older words may hold pixels that
// are no longer pending: that only costs a step that finds no seeds).
__device__ __forceinline__ uint32_t grow_tile(const HystScratch &hs, uint32_t t, const TileSeeds &sd, int lane,
                                              uint32_t p, const Facing &fp, bool rowwise = true,
                                              TileMasks *after = nullptr)
{
    const HystImage &im = sd.im;
    const int tx = sd.tx, ty = sd.ty;
    const bool hasL = tx > 0, hasR = tx < im.ntx - 1, hasU = ty > 0, hasD = ty < im.nty - 1;
    const uint32_t s_top = sd.top, s_bot = sd.bot, s_left = sd.left, s_right = sd.right;
    uint32_t e0 = ((s_left >> lane) & 1u) | (((s_right >> lane) & 1u) << 31);
    if (lane == 0) e0 |= s_top;
    if (lane == HT - 1) e0 |= s_bot;
    e0 &= p;
    const uint32_t e = flood_tile(e0, p, lane);

    // write the new edges and the shrunken pending set
    if (rowwise) {
        store_new_edges(im, tx, ty, lane, e);
    } else if (e) {
        uint8_t *row = im.map + (int64_t)(ty * HT + lane) * im.pitch + tx * HT;
        for (uint32_t bits = e; bits; bits &= bits - 1) row[__ffs(bits) - 1] = 255;
    }
    p &= ~e;
    hs.pend_bits[(size_t)t * HT + lane] = p;

    const uint32_t e_top = __shfl_sync(FULL, e, 0), e_bot = __shfl_sync(FULL, e, HT - 1);
    const uint32_t e_left = __ballot_sync(FULL, e & 1u), e_right = __ballot_sync(FULL, e >> 31);
    const uint32_t p_top = __shfl_sync(FULL, p, 0), p_bot = __shfl_sync(FULL, p, HT - 1);
    const uint32_t p_left = __ballot_sync(FULL, p & 1u), p_right = __ballot_sync(FULL, p >> 31);
    if (after) {
        // the border edges this step added and the border pixels left pending (every lane)
        after->edge_top = e_top; after->edge_bottom = e_bot; after->edge_left = e_left; after->edge_right = e_right;
        after->pend_top = p_top; after->pend_bottom = p_bot; after->pend_left = p_left; after->pend_right = p_right;
    }
    uint32_t aff = 0;
    if (lane == 0) {
        TileMasks *mt = &hs.masks[t];
        if (e_top) atomicOr(&mt->edge_top, e_top);
        if (e_bot) atomicOr(&mt->edge_bottom, e_bot);
        if (e_left) atomicOr(&mt->edge_left, e_left);
        if (e_right) atomicOr(&mt->edge_right, e_right);
        atomicAnd(&mt->pend_top, p_top);
        atomicAnd(&mt->pend_bottom, p_bot);
        atomicAnd(&mt->pend_left, p_left);
        atomicAnd(&mt->pend_right, p_right);
        // No fence: this warp reads these masks again only through lane 0 (the
        // thread that made these atomics) when it follows into a neighbour. A
        // warp of another CTA working on a neighbour at the same time may miss
        // these edges, but this warp checks that neighbour's pending border and
        // follows into it (a stale pending word only has more bits), so no seed
        // is lost; the end of the pass orders everything for the next one.
        // Neighbours whose facing border has pending pixels next to a new edge:
        if (hasU && e_top) {
            uint32_t d = e_top | (e_top << 1) | (e_top >> 1);
            if (fp.u & d) aff |= 1u << NB_U;
            if (hasL && (e_top & 1u) && (fp.ul >> 31)) aff |= 1u << NB_UL;
            if (hasR && (e_top >> 31) && (fp.ur & 1u)) aff |= 1u << NB_UR;
        }
        if (hasD && e_bot) {
            uint32_t d = e_bot | (e_bot << 1) | (e_bot >> 1);
            if (fp.d & d) aff |= 1u << NB_D;
            if (hasL && (e_bot & 1u) && (fp.dl >> 31)) aff |= 1u << NB_DL;
            if (hasR && (e_bot >> 31) && (fp.dr & 1u)) aff |= 1u << NB_DR;
        }
        if (hasL && e_left) {
            uint32_t d = e_left | (e_left << 1) | (e_left >> 1);
            if (fp.l & d) aff |= 1u << NB_L;
        }
        if (hasR && e_right) {
            uint32_t d = e_right | (e_right << 1) | (e_right >> 1);
            if (fp.r & d) aff |= 1u << NB_R;
        }
    }
    return __shfl_sync(FULL, aff, 0);
}

// ---------------------------------------------------------------- one launch per pass
// The pass of the one-launch-per-pass kernel (graph while-loops, the host-driven
// loop), whose CTAs need not all be resident at once (batches on several
// streams share the GPU): no warp waits for another. A warp that adds edges next to a
// neighbour's pending pixels follows them into that neighbour at once (depth
// first, up to CHASE_BUDGET tiles per worklist entry), so a chain of weak pixels
// across many tiles costs one pass, not one pass per tile; what the budget or
// the stack cannot take is queued for the next pass. A tile may be visited by
// two warps at a time: both only add edges, and each re-reads the masks, so the
// result is the same.
// One pass (all CTAs of the grid). The last CTA to finish swaps the worklists,
// counts the pass and sets keep_going (and, in a graph, the while-node's
// condition).
__device__ __forceinline__ void global_pass_stack(const HystScratch &hs, int in_graph, cudaGraphConditionalHandle cond,
                                            uint32_t (&stack)[WARPS][CHASE_STACK], uint32_t &visits)
{
    HystState *st = hs.state;
    const uint32_t k = *(volatile uint32_t *)&st->pass;
    const uint32_t cur = k & 1u, nxt = cur ^ 1u;
    uint32_t count = *(volatile uint32_t *)&st->list_count[cur];
    if (!CANNY_CHECK(count <= hs.max_tiles, &st->error)) count = hs.max_tiles;
    const int nimg = (int)st->nimg;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint32_t warp = (blockIdx.x * THREADS + threadIdx.x) >> 5;
    const uint32_t nwarps = gridDim.x * WARPS;
    const uint32_t *list = hs.lists + (size_t)cur * hs.max_tiles;
    const int chase_budget = st->chase_budget ? (int)st->chase_budget : STACK_BUDGET;
    if (threadIdx.x == 0) visits = 0;
    __syncthreads();
    uint32_t my_visits = 0;
    // each lane checks one worklist entry for seeds; the warp then grows the
    // tiles that have some, one after the other, and follows their chains
    for (uint32_t base = warp * 32u; base < count; base += nwarps * 32u) {
        const uint32_t i = base + (uint32_t)lane;
        uint32_t mine = 0;
        bool has = false;
        if (i < count) {
            TileSeeds sd;
            mine = __ldcg(&list[i]);      // (a cooperative launch reuses L1 across passes)
            has = CANNY_CHECK(mine < hs.max_tiles, &st->error) && find_seeds(hs, mine, nimg, sd);
        }
        my_visits += (lane == 0) ? min(32u, count - base) : 0u;   // entries examined
        uint32_t todo = __ballot_sync(FULL, has);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            uint32_t t = __shfl_sync(FULL, mine, src);
            int sp = 0, budget = chase_budget;
            for (;;) {
                TileSeeds sd;
                Facing fp;
                uint32_t aff = 0, ntx = 0;
                if (!CANNY_CHECK(t < hs.max_tiles, &st->error)) break;
                const uint32_t p_row = __ldcg(&hs.pend_bits[(size_t)t * HT + lane]);   // issued with the masks
                if (chase_seeds(hs, t, nimg, sd, lane, fp)) {
                    aff = grow_tile(hs, t, sd, lane, p_row, fp, false);
                    ntx = (uint32_t)sd.im.ntx;
                }
                ++my_visits;
                while (aff) {
                    const int d = __ffs(aff) - 1;
                    aff &= aff - 1;
                    const uint32_t n = neighbour(t, d, ntx);
                    if (sp < CHASE_STACK && budget > 0) {
                        if (lane == 0) stack[wl][sp] = n;
                        ++sp;
                        --budget;
                    } else if (lane == 0) {
                        push(hs, nxt, n, k + 2);
                    }
                }
                __syncwarp();
                if (sp == 0) break;
                t = stack[wl][--sp];
                __syncwarp();
            }
        }
    }
    if (lane == 0) atomicAdd(&visits, my_visits);

    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&st->visited, visits);
        __threadfence();
        if (atomicAdd(&st->done_ctas, 1u) == gridDim.x - 1) {
            __threadfence();
            const uint32_t next = atomicAdd(&st->list_count[nxt], 0u);
            st->list_count[cur] = 0;
            st->pass = k + 1;
            st->done_ctas = 0;
            bool more = next > 0;
            if (more && k + 1 >= st->max_passes) {
                st->error |= 1u;
                more = false;
            }
            st->keep_going = more ? 1u : 0u;
            __threadfence();
            if (in_graph) cudaGraphSetConditional(cond, more ? 1u : 0u);
        }
    }
}


// ---------------------------------------------------------------- the next step, read ahead
// Offsets (dx, dy) of the neighbour in direction d (NB_*).
__device__ __forceinline__ int nb_dx(int d) { return (int)((0x8861u >> (2 * d)) & 3u) - 1; }
__device__ __forceinline__ int nb_dy(int d) { return (int)((0x5A80u >> (2 * d)) & 3u) - 1; }

// Issued before a step's flood, so that the loads of the next step are in flight
// while it runs: lane k < 25 loads the masks of the tile at offset
// (k % 5 - 2, k / 5 - 2) from t (zero outside the image), every lane its row of
// the pending bitmap of each of t's eight neighbours (zero outside). The words
// may be older than the next step's start; a pending word only ever loses bits
// and an edge another warp adds next to a pending pixel is followed by that
// warp, so an older word costs at most a wasted step, never a missed seed.
__device__ __forceinline__ void read_ahead(const HystScratch &hs, const TileSeeds &sd, uint32_t t, int lane,
                                           TileMasks &blk, uint32_t (&pn)[8])
{
    const HystImage &im = sd.im;
    const int dx = lane % 5 - 2, dy = lane / 5 - 2;
    const int x = sd.tx + dx, y = sd.ty + dy;
    blk = TileMasks{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (lane < 25 && x >= 0 && x < im.ntx && y >= 0 && y < im.nty)
        blk = masks_cg(&hs.masks[(uint32_t)((int64_t)t + (int64_t)dy * im.ntx + dx)]);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int nx = sd.tx + nb_dx(d), ny = sd.ty + nb_dy(d);
        pn[d] = (nx >= 0 && nx < im.ntx && ny >= 0 && ny < im.nty)
                    ? __ldcg(&hs.pend_bits[(size_t)neighbour(t, d, (uint32_t)im.ntx) * HT + lane]) : 0u;
    }
}

// The seeds, facing pending words and pending row of t's neighbour in direction
// d0, from the words read ahead (every lane). t's own words are its masks after
// this step: the edges it had plus those the step added, and the pixels left
// pending.
__device__ __forceinline__ void step_ahead(TileSeeds &sd, Facing &fp, uint32_t &p_row, const TileMasks &blk,
                                           const uint32_t (&pn)[8], const TileMasks &after, int d0)
{
    const int ox = nb_dx(d0), oy = nb_dy(d0);
    enum { ET, EB, EL, ER, PT, PB, PL, PR };
    auto get = [&](int dx, int dy, int f) -> uint32_t {
        const int k = (dy + 2) * 5 + (dx + 2);
        const uint32_t w = f == ET ? blk.edge_top : f == EB ? blk.edge_bottom : f == EL ? blk.edge_left :
                           f == ER ? blk.edge_right : f == PT ? blk.pend_top : f == PB ? blk.pend_bottom :
                           f == PL ? blk.pend_left : blk.pend_right;
        uint32_t v = __shfl_sync(FULL, w, k);
        if (dx == 0 && dy == 0) {
            const uint32_t a = f == ET ? after.edge_top : f == EB ? after.edge_bottom : f == EL ? after.edge_left :
                               f == ER ? after.edge_right : f == PT ? after.pend_top : f == PB ? after.pend_bottom :
                               f == PL ? after.pend_left : after.pend_right;
            v = f < PT ? (v | a) : a;
        }
        return v;
    };
    const uint32_t pt = get(ox, oy, PT), pb = get(ox, oy, PB), pl = get(ox, oy, PL), pr = get(ox, oy, PR);
    const uint32_t eu = get(ox, oy - 1, EB), eul = get(ox - 1, oy - 1, EB), eur = get(ox + 1, oy - 1, EB);
    const uint32_t ed = get(ox, oy + 1, ET), edl = get(ox - 1, oy + 1, ET), edr = get(ox + 1, oy + 1, ET);
    const uint32_t el = get(ox - 1, oy, ER), er = get(ox + 1, oy, EL);
    fp.u = get(ox, oy - 1, PB); fp.ul = get(ox - 1, oy - 1, PB); fp.ur = get(ox + 1, oy - 1, PB);
    fp.d = get(ox, oy + 1, PT); fp.dl = get(ox - 1, oy + 1, PT); fp.dr = get(ox + 1, oy + 1, PT);
    fp.l = get(ox - 1, oy, PR); fp.r = get(ox + 1, oy, PL);
    sd.top = (eu | (eu << 1) | (eu >> 1) | (eul >> 31) | ((eur & 1u) << 31)) & pt;
    sd.bot = (ed | (ed << 1) | (ed >> 1) | (edl >> 31) | ((edr & 1u) << 31)) & pb;
    sd.left = dilate(el) & pl;
    sd.right = dilate(er) & pr;
    sd.tx += ox;
    sd.ty += oy;
#pragma unroll
    for (int d = 0; d < 8; ++d)
        if (d == d0) p_row = pn[d];
}

// ---------------------------------------------------------------- the in-pass queue
// (the cooperative kernel's passes: every CTA of its grid is resident, so a
// warp may wait for work that another warp queues)
// Work of one pass that any warp may take: a worklist entry found seeded while
// its warp was busy with another, or a branch of a chain (the neighbours a
// visit affected beyond the one its warp follows). Each item carries what is
// left of its chain's budget. q_open counts items queued but not yet finished
// plus CTAs whose warps are still on their worklist entries. A warp that queued
// an item stays until q_open is 0, so no item is left behind even if a CTA
// starts late (after others have left); the waiting warps keep taking branches
// while long chains run.
__device__ __forceinline__ unsigned long long make_item(uint32_t tag, uint32_t budget, uint32_t tile)
{
    return ((unsigned long long)tag << 48) | ((unsigned long long)budget << 32) | tile;
}

// Queue tile with budget (one thread). The caller has made its edges visible
// (a fence in every lane). A full queue hands the tile to the next pass instead.
__device__ __forceinline__ void queue_push(const HystScratch &hs, uint32_t tag, uint32_t budget, uint32_t tile,
                                           uint32_t nxt, uint32_t stamp)
{
    HystState *st = hs.state;
    atomicAdd(&st->q_open, 1u);
    const uint32_t slot = atomicAdd(&st->q_tail, 1u);
    if (slot < hs.max_tiles) {
        atomicExch(&hs.queue[slot], make_item(tag, budget, tile));
    } else {
        push(hs, nxt, tile, stamp);
        atomicSub(&st->q_open, 1u);
    }
}

// Take an item (lane 0): 0 if none is queued now. A claimed slot whose producer
// has not yet written it is waited for (bounded); on a timeout error bit 1 is
// set and the item is dropped (the run then reports the error).
__device__ __forceinline__ unsigned long long queue_pop(const HystScratch &hs, uint32_t tag)
{
    HystState *st = hs.state;
    for (;;) {
        const uint32_t h = *(volatile uint32_t *)&st->q_head;
        const uint32_t t = min(*(volatile uint32_t *)&st->q_tail, hs.max_tiles);
        if (h >= t) return 0ull;
        if (atomicCAS(&st->q_head, h, h + 1u) != h) continue;
        const uint64_t t0 = globaltimer_ns();
        for (;;) {
            const unsigned long long v = atomicExch(&hs.queue[h], 0ull);
            if ((uint32_t)(v >> 48) == tag) {
                __threadfence();                // the producer's edges before this warp reads masks
                return v;
            }
            // (v nonzero here is a leftover of a run that stopped on an error: dropped)
            if (globaltimer_ns() - t0 > WAIT_TIMEOUT_NS) {
                atomicOr(&st->error, 2u);
                atomicSub(&st->q_open, 1u);
                return 0ull;
            }
            __nanosleep(32);
        }
    }
}

// One pass over the current worklist, all CTAs of the grid. Warps take chunks
// of entries in order (32, or fewer when the list is short so that every warp
// gets some); the lanes check a chunk's entries for seeds at once. A warp grows
// a seeded tile and follows the chain it starts (depth first: it visits next a
// neighbour whose facing pending pixels touch the edges it added, while the
// chain's budget lasts); further affected neighbours, and on a short list the
// chunk's other seeded entries, go to the in-pass queue for idle warps, and
// what a spent budget or a full queue cannot take is listed for the next pass. A tile may be
// visited by two warps at a time: both only add edges, and each re-reads the
// masks, so the result is the same. The last CTA to finish swaps the
// worklists, counts the pass and sets keep_going (and, in a graph, the
// while-node's condition).
__device__ __forceinline__ void global_pass(const HystScratch &hs, int in_graph, cudaGraphConditionalHandle cond,
                                            uint32_t &visits, uint32_t &warps_on_list)
{
    HystState *st = hs.state;
    const uint32_t k = *(volatile uint32_t *)&st->pass;
    const uint32_t cur = k & 1u, nxt = cur ^ 1u;
    uint32_t count = *(volatile uint32_t *)&st->list_count[cur];
    if (!CANNY_CHECK(count <= hs.max_tiles, &st->error)) count = hs.max_tiles;
    const int nimg = (int)st->nimg;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * THREADS + threadIdx.x) >> 5;
    const uint32_t nwarps = gridDim.x * WARPS;
    const uint32_t *list = hs.lists + (size_t)cur * hs.max_tiles;
    const uint32_t budget0 = st->chase_budget ? st->chase_budget : (uint32_t)CHASE_BUDGET;
    const uint32_t tag = st->run_tag;
    const uint32_t chunk = count >= nwarps * 32u ? 32u : max(1u, (count + nwarps - 1u) / nwarps);
    if (threadIdx.x == 0) {
        visits = 0;
        warps_on_list = WARPS;
        atomicAdd(&st->q_open, 1u);            // the CTA keeps the pass open while its warps work the list
    }
    __syncthreads();
    uint32_t my_visits = 0;
    bool pushed = false;                       // this thread queued an item

    // follow the chain from tile t with budget b (whole warp); the words of the
    // step that follows a step are read during its flood
    auto chase = [&](uint32_t t, uint32_t b) {
        TileSeeds sd;
        Facing fp;
        uint32_t p_row = 0u;
        bool ahead = false;                    // sd, fp and p_row of t are already known
        for (;;) {
            uint32_t aff = 0, ntx = 0;
            if (!CANNY_CHECK(t < hs.max_tiles, &st->error)) return;
            bool has;
            if (ahead) {
                has = (sd.top | sd.bot | sd.left | sd.right) != 0u;
            } else {
                p_row = __ldcg(&hs.pend_bits[(size_t)t * HT + lane]);   // issued with the masks
                has = chase_seeds(hs, t, nimg, sd, lane, fp);
            }
            ahead = false;
            TileMasks blk, after;
            uint32_t pn[8];
            if (has) {
                read_ahead(hs, sd, t, lane, blk, pn);
                aff = grow_tile(hs, t, sd, lane, p_row, fp, true, &after);
                ntx = (uint32_t)sd.im.ntx;
            }
            ++my_visits;
            if (!aff) return;
            // the first affected neighbour is followed by this warp (lane 0 made
            // the mask updates it reads back); the others are handed on
            const int d0 = __ffs(aff) - 1;
            aff &= aff - 1;
            const uint32_t next = neighbour(t, d0, ntx);
            if (aff && b > 0) {
                __threadfence();                    // this visit's edges, before another warp looks
                __syncwarp();
            }
            if (lane == 0) {
                while (aff) {
                    const int d = __ffs(aff) - 1;
                    aff &= aff - 1;
                    const uint32_t n = neighbour(t, d, ntx);
                    if (b > 0) {
                        queue_push(hs, tag, b - 1u, n, nxt, k + 2);
                        pushed = true;
                    } else {
                        push(hs, nxt, n, k + 2);
                    }
                }
            }
            __syncwarp();
            if (b == 0) {
                if (lane == 0) push(hs, nxt, next, k + 2);
                return;
            }
            step_ahead(sd, fp, p_row, blk, pn, after, d0);
            ahead = true;
            t = next;
            --b;
        }
    };

    // worklist chunks, spread over the warps in order
    for (uint32_t base = warp * chunk; base < count; base += nwarps * chunk) {
        const uint32_t i = base + (uint32_t)lane;
        uint32_t mine = 0;
        bool has = false;
        if ((uint32_t)lane < chunk && i < count) {
            TileSeeds sd;
            mine = __ldcg(&list[i]);      // (a cooperative launch reuses L1 across passes)
            has = CANNY_CHECK(mine < hs.max_tiles, &st->error) && find_seeds(hs, mine, nimg, sd);
        }
        my_visits += (lane == 0) ? min(chunk, count - base) : 0u;   // entries examined
        uint32_t todo = __ballot_sync(FULL, has);
        if (todo && chunk < 32u) {
            // a short list leaves warps idle: the other seeded entries go to them
            // (nothing of this warp's to publish)
            const int src = __ffs(todo) - 1;
            if (has && lane != src) {
                queue_push(hs, tag, budget0, mine, nxt, k + 2);
                pushed = true;
            }
            todo = 1u << src;
        }
        // a long list keeps every warp busy: the warp grows its seeded entries in turn
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            chase(__shfl_sync(FULL, mine, src), budget0);
        }
    }
    // the CTA's last warp off the list releases its hold on the pass
    if (lane == 0 && atomicSub(&warps_on_list, 1u) == 1u) atomicSub(&st->q_open, 1u);

    // queued items until every item of the pass is finished. Warps that queued
    // some stay; of the others at most as many wait as the grid has CTAs (more
    // pollers of the control block slow the warps that work).
    bool waiter = __any_sync(FULL, pushed);
    if (lane == 0 && !waiter) waiter = atomicAdd(&st->q_waiters, 1u) < gridDim.x;
    if (__shfl_sync(FULL, waiter, 0)) {
        const uint64_t t0 = globaltimer_ns();
        uint32_t nap = 32;
        for (;;) {
            unsigned long long item = 0;
            bool done = false;
            if (lane == 0) {
                item = queue_pop(hs, tag);
                if (!item) {
                    const bool late = globaltimer_ns() - t0 > WAIT_TIMEOUT_NS;
                    done = *(volatile uint32_t *)&st->q_open == 0u || (*(volatile uint32_t *)&st->error & 2u) ||
                           late;
                    if (late && *(volatile uint32_t *)&st->q_open != 0u) atomicOr(&st->error, 2u);
                }
            }
            item = __shfl_sync(FULL, item, 0);
            if (item) {
                __threadfence();
                chase((uint32_t)item, (uint32_t)(item >> 32) & 0xffffu);
                if (lane == 0) atomicSub(&st->q_open, 1u);
                nap = 32;
                continue;
            }
            if (__shfl_sync(FULL, done, 0)) break;
            __nanosleep(nap);
            nap = min(nap * 2u, 1024u);
        }
    }
    if (lane == 0) atomicAdd(&visits, my_visits);

    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&st->visited, visits);
        __threadfence();
        if (atomicAdd(&st->done_ctas, 1u) == gridDim.x - 1) {
            __threadfence();
            const uint32_t next = atomicAdd(&st->list_count[nxt], 0u);
            st->list_count[cur] = 0;
            st->uf_entries = count;           // a union-find stage after this pass labels these tiles
            st->uf_count = 0;
            st->q_head = st->q_tail = 0;
            st->q_open = st->q_waiters = 0;
            st->pass = k + 1;
            st->done_ctas = 0;
            bool more = next > 0;
            if (more && k + 1 >= st->max_passes) {
                st->error |= 1u;
                more = false;
            }
            if (st->error & 2u) more = false;
            st->keep_going = more ? 1u : 0u;
            __threadfence();
            if (in_graph) cudaGraphSetConditional(cond, more ? 1u : 0u);
        }
    }
}

__global__ void __launch_bounds__(THREADS)
hyst_global_kernel(HystScratch hs, int in_graph, cudaGraphConditionalHandle cond)
{
    __shared__ uint32_t stack[WARPS][CHASE_STACK];
    __shared__ uint32_t visits;
    global_pass_stack(hs, in_graph, cond, stack, visits);
}

// Grid-wide barrier of a cooperative launch (every CTA is resident): the last
// CTA to arrive advances the generation. The wait is bounded; if it runs out,
// error bit 1 is set and false returned in every thread of the CTA.

__device__ __forceinline__ bool grid_barrier(HystState *st)
{
    __shared__ uint32_t ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ok = 1;
        const uint32_t gen = atomicAdd(&st->bar_gen, 0u);      // read before arriving
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            // bounded by time: a legitimate pass of the largest image ends within
            // milliseconds, so a second without the last arrival is a failure
            const uint64_t t0 = globaltimer_ns();
            while (atomicAdd(&st->bar_gen, 0u) == gen) {
                if (globaltimer_ns() - t0 > WAIT_TIMEOUT_NS) {
                    atomicOr(&st->error, 2u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------- long chains: union-find
// When the first pass leaves work for a second one (a chain longer than the
// chase budget, or a full in-pass queue), the rest is resolved at once instead
// of pass after pass. Every pending pixel is, by then,
// a weak pixel not connected inside its tile to an edge, so a pending pixel
// becomes an edge exactly when it is connected, through pending pixels across
// tile borders, to a pending border pixel next to an edge of a neighbouring tile.
//   label   each tile with pending border pixels splits them into the components
//           of its pending pixels (one flood per component) and lists itself;
//   union   each listed tile joins its components with those of its right,
//           lower and two lower diagonal neighbours wherever pending border
//           pixels touch (lock-free union-find, links by atomicCAS, finds with
//           path halving), and marks components next to a neighbour's edge;
//   roots   a marked component marks its root (a find with path halving);
//   apply   each listed tile floods its pending pixels from the border pixels
//           whose component's root is marked and writes the new edges.
// Four phases separated by grid barriers, whatever the chain length. Links go
// from the larger root to the smaller and every find halves the path it walks,
// so the trees stay shallow (the finds of the roots phase shorten them again
// for the apply phase).
constexpr int UF_LSTRIDE = 128;         // label bytes a tile: 124 border pixels, count at byte 127
constexpr int UF_COUNT = 127;
constexpr uint32_t UF_MAXC = 64;        // components a tile (at most 62 can touch its border)

// Border pixel (x, y) of a tile as a position: 0..31 top row, 32..63 bottom row,
// 64..93 left column rows 1..30, 94..123 right column rows 1..30.
__device__ __forceinline__ int border_pos(int x, int y)
{
    return y == 0 ? x : (y == HT - 1 ? HT + x : (x == 0 ? 2 * HT + y - 1 : 3 * HT - 2 + y - 1));
}

__device__ __forceinline__ bool pending_border(const TileMasks &m)
{
    return (m.pend_top | m.pend_bottom | m.pend_left | m.pend_right) != 0u;
}

__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x)
{
    for (;;) {
        const uint32_t p = __ldcg(parent + x);
        if (p == x) return x;
        const uint32_t gp = __ldcg(parent + p);
        if (gp != p) parent[x] = gp;          // path halving: gp is an ancestor of x
        x = gp;
    }
}

__device__ __forceinline__ void uf_union(uint32_t *parent, uint32_t a, uint32_t b)
{
    for (;;) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a < b) { const uint32_t t = a; a = b; b = t; }
        if (atomicCAS(parent + a, a, b) == a) return;   // link the larger root under the smaller
    }
}

__device__ __forceinline__ uint32_t uf_comp(const HystScratch &hs, uint32_t t, int pos)
{
    return t * UF_MAXC + __ldcg(hs.uf_label + (size_t)t * UF_LSTRIDE + pos);
}

// label: every tile with pending border pixels, one warp a tile. The stage runs
// right after the first pass, whose worklist (list 0) holds every tile the local
// fill left with pending border pixels (pending pixels only ever become edges),
// so that list is the one to scan; the labelled tiles are listed in list 1.
__device__ __forceinline__ void uf_label_phase(const HystScratch &hs, int lane, uint32_t warp, uint32_t nwarps)
{
    HystState *st = hs.state;
    // every tile with pending border pixels now was on the first pass's worklist
    // (list 0: the tiles the local fill left with pending border pixels)
    const uint32_t n0 = min(*(volatile uint32_t *)&st->uf_entries, hs.max_tiles);
    uint32_t *uf_list = hs.lists + hs.max_tiles;
    for (uint32_t i = warp; i < n0; i += nwarps) {
        const uint32_t t = __ldcg(&hs.lists[i]);
        if (!CANNY_CHECK(t < hs.max_tiles, &st->error)) continue;
        const TileMasks m = masks_cg(&hs.masks[t]);
        if (!pending_border(m)) continue;
        {
            const uint32_t P = __ldcg(&hs.pend_bits[(size_t)t * HT + lane]);
            uint8_t *lab = hs.uf_label + (size_t)t * UF_LSTRIDE;
            uint32_t rt = m.pend_top, rb = m.pend_bottom;
            uint32_t rl = m.pend_left & 0x7FFFFFFEu, rr = m.pend_right & 0x7FFFFFFEu;   // rows 1..30
            uint32_t k = 0;
            while ((rt | rb | rl | rr) != 0u && k < UF_MAXC) {
                int sy, sx;
                if (rt) { sy = 0; sx = __ffs(rt) - 1; }
                else if (rb) { sy = HT - 1; sx = __ffs(rb) - 1; }
                else if (rl) { sy = __ffs(rl) - 1; sx = 0; }
                else { sy = __ffs(rr) - 1; sx = HT - 1; }
                const uint32_t C = flood_tile(lane == sy ? (1u << sx) : 0u, P, lane);
                const uint32_t ct = __shfl_sync(FULL, C, 0), cb = __shfl_sync(FULL, C, HT - 1);
                const uint32_t cl = __ballot_sync(FULL, C & 1u), cr = __ballot_sync(FULL, C >> 31);
                if (((ct & rt) >> lane) & 1u) lab[lane] = (uint8_t)k;
                if (((cb & rb) >> lane) & 1u) lab[HT + lane] = (uint8_t)k;
                if (((cl & rl) >> lane) & 1u) lab[2 * HT + lane - 1] = (uint8_t)k;
                if (((cr & rr) >> lane) & 1u) lab[3 * HT - 2 + lane - 1] = (uint8_t)k;
                rt &= ~ct;
                rb &= ~cb;
                rl &= ~cl;
                rr &= ~cr;
                if (lane == 0) {
                    hs.uf_parent[(size_t)t * UF_MAXC + k] = t * UF_MAXC + k;
                    hs.uf_seeded[(size_t)t * UF_MAXC + k] = 0;
                }
                ++k;
            }
            if (lane == 0) {
                lab[UF_COUNT] = (uint8_t)k;
                const uint32_t slot = atomicAdd(&st->uf_count, 1u);
                if (CANNY_CHECK(slot < hs.max_tiles, &st->error)) uf_list[slot] = t;
            }
        }
    }
}

// union: a listed tile with its right, lower, lower-right and lower-left neighbours;
// components next to a neighbour's edge are marked
__device__ __forceinline__ void uf_union_phase(const HystScratch &hs, int lane, uint32_t warp, uint32_t nwarps)
{
    HystState *st = hs.state;
    const uint32_t n = min(*(volatile uint32_t *)&st->uf_count, hs.max_tiles);
    const int nimg = (int)st->nimg;
    for (uint32_t i = warp; i < n; i += nwarps) {
        const uint32_t t = __ldcg(&hs.lists[hs.max_tiles + i]);
        TileSeeds sd;
        find_seeds(hs, t, nimg, sd);
        const HystImage &im = sd.im;
        const int tx = sd.tx, ty = sd.ty;
        const uint32_t ntx = (uint32_t)im.ntx;
        const bool hasL = tx > 0, hasR = tx < im.ntx - 1, hasD = ty < im.nty - 1;
        const TileMasks m = masks_cg(&hs.masks[t]);
        const int y = lane, x = lane;
        // marks: pending border pixels next to an edge of a neighbouring tile
        if ((sd.top >> x) & 1u) hs.uf_seeded[uf_comp(hs, t, x)] = 1;
        if ((sd.bot >> x) & 1u) hs.uf_seeded[uf_comp(hs, t, HT + x)] = 1;
        if ((sd.left >> y) & 1u) hs.uf_seeded[uf_comp(hs, t, border_pos(0, y))] = 1;
        if ((sd.right >> y) & 1u) hs.uf_seeded[uf_comp(hs, t, border_pos(HT - 1, y))] = 1;
        if (hasR && ((m.pend_right >> y) & 1u)) {
            const uint32_t nb = t + 1;
            const uint32_t pl = __ldcg(&hs.masks[nb].pend_left);
            for (int dy = -1; dy <= 1; ++dy) {
                const int y2 = y + dy;
                if (y2 >= 0 && y2 < HT && ((pl >> y2) & 1u))
                    uf_union(hs.uf_parent, uf_comp(hs, t, border_pos(HT - 1, y)), uf_comp(hs, nb, border_pos(0, y2)));
            }
        }
        if (hasD && ((m.pend_bottom >> x) & 1u)) {
            const uint32_t nb = t + ntx;
            const uint32_t pt = __ldcg(&hs.masks[nb].pend_top);
            for (int dx = -1; dx <= 1; ++dx) {
                const int x2 = x + dx;
                if (x2 >= 0 && x2 < HT && ((pt >> x2) & 1u))
                    uf_union(hs.uf_parent, uf_comp(hs, t, HT + x), uf_comp(hs, nb, x2));
            }
        }
        if (lane == 0 && hasD && hasR && (m.pend_bottom >> 31) && (__ldcg(&hs.masks[t + ntx + 1].pend_top) & 1u))
            uf_union(hs.uf_parent, uf_comp(hs, t, 2 * HT - 1), uf_comp(hs, t + ntx + 1, 0));
        if (lane == 1 && hasD && hasL && (m.pend_bottom & 1u) && (__ldcg(&hs.masks[t + ntx - 1].pend_top) >> 31))
            uf_union(hs.uf_parent, uf_comp(hs, t, HT), uf_comp(hs, t + ntx - 1, HT - 1));
    }
}

// roots: a marked component marks its root
__device__ __forceinline__ void uf_roots_phase(const HystScratch &hs, int lane, uint32_t warp, uint32_t nwarps)
{
    HystState *st = hs.state;
    const uint32_t n = min(*(volatile uint32_t *)&st->uf_count, hs.max_tiles);
    for (uint32_t i = warp; i < n; i += nwarps) {
        const uint32_t t = __ldcg(&hs.lists[hs.max_tiles + i]);
        const uint32_t k = __ldcg(hs.uf_label + (size_t)t * UF_LSTRIDE + UF_COUNT);
        for (uint32_t j = (uint32_t)lane; j < k; j += 32u) {
            const uint32_t c = t * UF_MAXC + j;
            if (__ldcg(hs.uf_seeded + c)) hs.uf_seeded[uf_find(hs.uf_parent, c)] = 1;
        }
    }
}

// apply: a listed tile floods its pending pixels from the border pixels of marked
// components and writes the new edges
__device__ __forceinline__ void uf_apply_phase(const HystScratch &hs, int lane, uint32_t warp, uint32_t nwarps)
{
    HystState *st = hs.state;
    const uint32_t n = min(*(volatile uint32_t *)&st->uf_count, hs.max_tiles);
    const int nimg = (int)st->nimg;
    for (uint32_t i = warp; i < n; i += nwarps) {
        const uint32_t t = __ldcg(&hs.lists[hs.max_tiles + i]);
        const TileMasks m = masks_cg(&hs.masks[t]);
        const int y = lane, x = lane;
        auto marked = [&](int pos) { return __ldcg(hs.uf_seeded + uf_find(hs.uf_parent, uf_comp(hs, t, pos))) != 0; };
        const bool st_top = ((m.pend_top >> x) & 1u) && marked(x);
        const bool st_bot = ((m.pend_bottom >> x) & 1u) && marked(HT + x);
        const bool st_l = y > 0 && y < HT - 1 && ((m.pend_left >> y) & 1u) && marked(border_pos(0, y));
        const bool st_r = y > 0 && y < HT - 1 && ((m.pend_right >> y) & 1u) && marked(border_pos(HT - 1, y));
        const uint32_t top = __ballot_sync(FULL, st_top), bot = __ballot_sync(FULL, st_bot);
        uint32_t e0 = (st_l ? 1u : 0u) | (st_r ? 0x80000000u : 0u);
        if (lane == 0) e0 |= top;
        if (lane == HT - 1) e0 |= bot;
        if (!__any_sync(FULL, e0 != 0u)) continue;
        const uint32_t p = __ldcg(&hs.pend_bits[(size_t)t * HT + lane]);
        const uint32_t e = flood_tile(e0 & p, p, lane);
        const HystImage im = hs.imgs[find_image(hs.imgs, nimg, t)];
        const uint32_t local = t - im.tile_base;
        const int tx = (int)(local % (uint32_t)im.ntx), ty = (int)(local / (uint32_t)im.ntx);
        store_new_edges(im, tx, ty, lane, e);
        hs.pend_bits[(size_t)t * HT + lane] = p & ~e;
    }
}

// The four phases in one cooperative launch (every CTA resident); false if a
// barrier's bounded wait ran out.
__device__ __forceinline__ bool uf_resolve(const HystScratch &hs)
{
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * THREADS + threadIdx.x) >> 5, nwarps = gridDim.x * WARPS;
    // (uf_count and uf_entries were set by the last CTA of the pass)
    uf_label_phase(hs, lane, warp, nwarps);
    if (!grid_barrier(hs.state)) return false;
    uf_union_phase(hs, lane, warp, nwarps);
    if (!grid_barrier(hs.state)) return false;
    uf_roots_phase(hs, lane, warp, nwarps);
    if (!grid_barrier(hs.state)) return false;
    uf_apply_phase(hs, lane, warp, nwarps);
    if (!grid_barrier(hs.state)) return false;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        HystState *st = hs.state;
        st->visited += st->uf_count;
        st->pass += 1;                          // the union-find stage counts as one pass
        st->keep_going = 0;
        st->list_count[0] = st->list_count[1] = 0;
    }
    return true;
}

// All passes in one cooperative launch: pass, barrier, stop when the last CTA
// of the pass found nothing more to do (or the pass cap was reached).
__global__ void __launch_bounds__(THREADS, 2)
hyst_global_coop_kernel(HystScratch hs)
{
    __shared__ uint32_t visits, warps_on_list;
    for (;;) {
        global_pass(hs, 0, cudaGraphConditionalHandle{}, visits, warps_on_list);
        if (!grid_barrier(hs.state)) break;
        if (!*(volatile uint32_t *)&hs.state->keep_going) break;
        // work left after the first pass: resolve every long chain at once
        if (hs.uf_parent && *(volatile uint32_t *)&hs.state->pass == 1u &&
            *(volatile uint32_t *)&hs.state->uf_entries <= UF_MAX_ENTRIES) {
            uf_resolve(hs);
            break;
        }
    }
}

__global__ void hyst_init_kernel(HystState *st, uint32_t ntiles, uint32_t nimg, uint32_t max_passes,
                                 HystImage *imgs, HystImage single, int write_single, uint32_t chase_budget)
{
    if (write_single) imgs[0] = single;
    HystState s = {};
    s.run_tag = st->run_tag % 65535u + 1u;
    s.ntiles = ntiles;
    s.nimg = nimg;
    s.max_passes = max_passes;
    s.chase_budget = chase_budget;
    s.keep_going = 1;
    *st = s;
}

__global__ void hyst_init_from_header_kernel(HystState *st, const BatchHeader *hdr)
{
    HystState s = {};
    s.run_tag = st->run_tag % 65535u + 1u;
    s.ntiles = hdr->ntiles;
    s.nimg = hdr->nimg;
    s.max_passes = hdr->max_passes;
    s.chase_budget = hdr->chase_budget;
    s.keep_going = 1;
    *st = s;
}

// OR a run's error bits into an accumulator that outlives the next reset.
__global__ void hyst_error_or_kernel(const HystState *st, uint32_t *acc)
{
    const uint32_t e = st->error;
    if (e) atomicOr(acc, e);
}

}  // namespace

// Per device (cached): CTAs of a global pass, and whether one cooperative launch
// of that grid fits.
namespace {
constexpr int MAX_DEVICES = 64;
int g_grid[MAX_DEVICES] = {};
int g_coop[MAX_DEVICES] = {};       // 0: not yet known, 1: no, 2: yes
int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) dev = 0;
    return dev;
}
}  // namespace

int hyst_pass_grid()
{
    const int dev = current_device();
    if (!g_grid[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        g_grid[dev] = 2 * sms;
    }
    return g_grid[dev];
}

cudaError_t hyst_reset(const HystScratch &hs, uint32_t ntiles, uint32_t nimg, uint32_t max_passes,
                       cudaStream_t s, const HystImage *single, uint32_t chase_budget)
{
    // the worklist stamps need no clearing: the local fill writes every tile's stamp
    HystImage one = single ? *single : HystImage{};
    hyst_init_kernel<<<1, 1, 0, s>>>(hs.state, ntiles, nimg, max_passes, hs.imgs, one, single ? 1 : 0,
                                     chase_budget);
    return cudaGetLastError();
}

cudaError_t launch_hyst_local_single(const HystScratch &hs, HystImage img, cudaStream_t s)
{
    uint32_t ntiles = (uint32_t)img.ntx * (uint32_t)img.nty;
    if (ntiles == 0) return cudaSuccess;
    int grid = (int)((ntiles + WARPS - 1) / WARPS);
    hyst_local_kernel<true><<<grid, THREADS, 0, s>>>(hs, img, ntiles, 1);
    return cudaGetLastError();
}

cudaError_t launch_hyst_local_batch(const HystScratch &hs, uint32_t ntiles, uint32_t nimg, cudaStream_t s)
{
    if (ntiles == 0) return cudaSuccess;
    int grid = (int)((ntiles + WARPS - 1) / WARPS);
    HystImage none = {};
    hyst_local_kernel<false><<<grid, THREADS, 0, s>>>(hs, none, ntiles, nimg);
    return cudaGetLastError();
}

cudaError_t launch_hyst_global_pass(const HystScratch &hs, int grid, bool in_graph,
                                    unsigned long long cond_handle, cudaStream_t s)
{
    hyst_global_kernel<<<grid, THREADS, 0, s>>>(hs, in_graph ? 1 : 0,
                                                (cudaGraphConditionalHandle)cond_handle);
    return cudaGetLastError();
}

bool hyst_coop_supported()
{
    const int dev = current_device();
    if (g_coop[dev] == 0) {
        int coop = 0, per_sm = 0, sms = 0;
        const bool ok = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
                        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hyst_global_coop_kernel, THREADS,
                                                                      0) == cudaSuccess &&
                        (int64_t)per_sm * sms >= hyst_pass_grid();
        cudaGetLastError();
        g_coop[dev] = ok ? 2 : 1;
    }
    return g_coop[dev] == 2;
}

namespace {
// Test hook: arrivals at the cooperative passes' grid barrier that no CTA
// makes, more than any grid has CTAs, so no arrival ever completes the barrier.
__global__ void hyst_phantom_arrival_kernel(HystState *st) { atomicAdd(&st->bar_count, 1u << 30); }
}  // namespace

cudaError_t launch_hyst_phantom_arrival(const HystScratch &hs, cudaStream_t s)
{
    hyst_phantom_arrival_kernel<<<1, 1, 0, s>>>(hs.state);
    return cudaGetLastError();
}

cudaError_t launch_hyst_global_coop(const HystScratch &hs, cudaStream_t s, uint32_t ntiles)
{
    if (!hyst_coop_supported()) return cudaErrorNotSupported;
    HystScratch hs_copy = hs;
    void *args[] = {&hs_copy};
    // a small image needs fewer CTAs (a warp per tile at most), and every pass's
    // end and grid barrier costs an arrival per CTA
    int grid = hyst_pass_grid();
    if (ntiles > 0) grid = (int)std::min<uint64_t>((uint64_t)grid, std::max<uint64_t>(4, ((uint64_t)ntiles + WARPS - 1) / WARPS));
    return cudaLaunchCooperativeKernel((void *)hyst_global_coop_kernel, dim3(grid), dim3(THREADS), args, 0, s);
}

// Append { while (cond) hyst_global_kernel } to graph g after the given nodes.
cudaError_t hyst_add_loop(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out)
{
    cudaGraphConditionalHandle cond;
    cudaError_t err = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
    if (err != cudaSuccess) return err;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    err = cudaGraphAddNode(out, g, deps, nullptr, ndeps, &cp);
    if (err != cudaSuccess) return err;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    HystScratch hs_copy = hs;
    int in_graph = 1;
    void *args[] = {&hs_copy, &in_graph, &cond};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)hyst_global_kernel;
    kp.gridDim = dim3(hyst_pass_grid());
    kp.blockDim = dim3(THREADS);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t knode;
    return cudaGraphAddKernelNode(&knode, body, nullptr, 0, &kp);
}

cudaError_t hyst_add_coop(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out)
{
    if (!hyst_coop_supported()) return cudaErrorNotSupported;
    HystScratch hs_copy = hs;
    void *args[] = {&hs_copy};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)hyst_global_coop_kernel;
    kp.gridDim = dim3(hyst_pass_grid());
    kp.blockDim = dim3(THREADS);
    kp.kernelParams = args;
    cudaError_t err = cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
    if (err != cudaSuccess) return err;
    cudaKernelNodeAttrValue v = {};
    v.cooperative = 1;
    return cudaGraphKernelNodeSetAttribute(*out, cudaLaunchAttributeCooperative, &v);
}

// Append { *acc |= state->error } to graph g after the given nodes.
cudaError_t hyst_add_error_or(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                              uint32_t *acc, cudaGraphNode_t *out)
{
    const HystState *st = hs.state;
    void *args[] = {(void *)&st, (void *)&acc};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)hyst_error_or_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

// Append the control-block reset that reads its sizes from a batch header.
cudaError_t hyst_add_init_from_header(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                                      const HystScratch &hs, const BatchHeader *hdr, cudaGraphNode_t *out)
{
    HystState *st = hs.state;
    const BatchHeader *h = hdr;
    void *args[] = {&st, &h};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)hyst_init_from_header_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

// Build the executable graph { while (cond) hyst_global_kernel } for this scratch.
cudaError_t hyst_build_graph(const HystScratch &hs, cudaGraph_t *graph_out, cudaGraphExec_t *exec_out)
{
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaError_t err = cudaGraphCreate(&g, 0);
    if (err != cudaSuccess) return err;
    cudaGraphNode_t loop;
    err = hyst_add_loop(g, nullptr, 0, hs, &loop);
    if (err == cudaSuccess) err = cudaGraphInstantiate(&ex, g, 0);
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return err;
    }
    *graph_out = g;
    *exec_out = ex;
    return cudaSuccess;
}

}  // namespace canny
