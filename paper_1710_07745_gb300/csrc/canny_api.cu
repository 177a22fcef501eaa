// canny_api.cu -- the C ABI of libcanny (declared in include/canny.h): argument
// checks, context scratch, and the launch sequence of the pipeline
//   stencil (Steps 1-3 + thresholds) -> local fill -> global passes (Step 4).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "canny_internal.cuh"

using namespace canny;

struct canny_ctx {
    int max_w = 0, max_h = 0;
    canny_params p = {};
    IntThresholds it = {};
    FloatParams fp = {};

    HystScratch hs = {};
    void *hyst_mem = nullptr;          // one allocation for the hysteresis scratch
    float *mag = nullptr;              // float path: strength after suppression
    float *d_max = nullptr;            // float path: the image's largest strength
    void *fmaps = nullptr;             // float path: squared strengths + sectors (pass 1 -> pass 2)
    size_t fmaps_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int use_graph = 1;                 // 0 after a graph could not be built: host-driven passes
    uint32_t *h_state = nullptr;       // pinned copy of the device control block

    uint8_t *d_host_in = nullptr, *d_host_out = nullptr;   // buffers of canny_run_host

    HystImage *h_imgs = nullptr;       // pinned staging for batch descriptors
    uint32_t h_imgs_cap = 0;
    cudaEvent_t staging_free = nullptr;

    cudaStream_t last_stream = nullptr;
    canny_stats last = {};

    // per-stage timing: EV_PER_RUN events per timed run
    int timing = 0;
    std::vector<cudaEvent_t> ev;
    int ev_runs = 0;

    // launch configuration of the fused kernel (canny_set_tuning / canny_autotune_batch)
    int band = 0;                      // rows per unit of work; 0: chosen per image size
    int ctas_per_sm = 0;               // batches: 0 = one CTA per unit, else persistent CTAs per SM
    int direct_loads = 0;              // 1: inputs the TMA path cannot read are not repitched
    int chase_budget = 0;              // global passes: tiles one worklist entry may chase (0: default)
    int batch_passes = 0;              // batch graphs: 0 = while-loop of passes, 1 = one cooperative node

    // integer-path batches: per staging slot one graph per fused-kernel variant
    // ([0] TMA or direct loads per image, [1] TMA only), descriptors uploaded
    // from pinned memory
    struct Slot {
        unsigned char *h_blob = nullptr;
        cudaGraph_t graph[2] = {nullptr, nullptr};
        cudaGraphExec_t exec[2] = {nullptr, nullptr};
        cudaGraphNode_t k1node[2] = {nullptr, nullptr};   // the fused kernel's node (grid set per launch)
        cudaEvent_t done = nullptr;
        bool valid[2] = {false, false};   // graph matches the current scratch and configuration
    } slots[2];
    int next_slot = 0;
    unsigned char *d_blob = nullptr;   // BatchHeader + BatchImage[cap] + CUtensorMap[cap] + Repitch[cap]

    // 16-byte pitched copies of inputs the TMA path cannot read (single image / batch)
    uint8_t *d_stage = nullptr, *d_bstage = nullptr;
    size_t stage_cap = 0, bstage_cap = 0;
    uint32_t blob_cap = 0;
    std::unordered_map<std::string, CUtensorMap> tmaps;   // encoded input maps, by (pointer, size, pitch)

    // frame sequences (canny_run_frames): two device slots, each with a graph of one
    // frame's whole pipeline; uploads and downloads run on streams of their own
    struct FrameSlot {
        uint8_t *d_in = nullptr, *d_out = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t up = nullptr, comp = nullptr, down = nullptr;
    } fslots[2];
    int frame_w = 0, frame_h = 0, frame_pitch = 0;   // size the slot buffers hold; graphs valid if exec set
    cudaStream_t s_up = nullptr, s_down = nullptr, s_cap = nullptr;
    cudaEvent_t frame_start = nullptr;
    uint32_t *d_frame_err = nullptr;                  // OR of the frames' hysteresis error bits
};

namespace {

constexpr int EV_PER_RUN = 5;   // before reset, after reset, after stencil, after local fill, after global

canny_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return CANNY_OK;
    if (e == cudaErrorMemoryAllocation) return CANNY_ENOMEM;
    return CANNY_ECUDA;
}

bool is_int_valued(float v) { return v == floorf(v); }

canny_status check_params(const canny_params *p)
{
    if (!p) return CANNY_EINVAL;
    if (p->path != CANNY_PATH_INT && p->path != CANNY_PATH_F32) return CANNY_EINVAL;
    if (!(p->low >= 0.f) || !(p->high >= 0.f) || !(p->low <= p->high)) return CANNY_EINVAL;
    if (p->max_passes < 0) return CANNY_EINVAL;
    if (p->path == CANNY_PATH_INT) {
        if (!is_int_valued(p->low) || !is_int_valued(p->high) || p->high >= 32768.f) return CANNY_EINVAL;
    } else {
        if (!(p->sigma > 0.f) || p->ksize < 3 || p->ksize > MAX_KSIZE || (p->ksize % 2) == 0)
            return CANNY_EINVAL;
    }
    return CANNY_OK;
}

uint32_t tiles_of(int w, int h)
{
    if (w <= 0 || h <= 0) return 0;
    return (uint32_t)((w + HT - 1) / HT) * (uint32_t)((h + HT - 1) / HT);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Failures injected by canny_inject_faults (test hooks).
std::atomic<int> g_fail_device{0}, g_fail_arena{0}, g_fail_barrier{0}, g_host_passes{0};

bool take_failure(std::atomic<int> &n)
{
    int v = n.load();
    while (v > 0)
        if (n.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

// Frame graphs hold the scratch pointers and the band height: dropped with the batch graphs.
void drop_frame_graphs(canny_ctx *c)
{
    for (auto &f : c->fslots) {
        if (f.exec) cudaGraphExecDestroy(f.exec);
        if (f.graph) cudaGraphDestroy(f.graph);
        f.exec = nullptr;
        f.graph = nullptr;
    }
}

void free_frames(canny_ctx *c)
{
    drop_frame_graphs(c);
    for (auto &f : c->fslots) {
        if (f.d_in) cudaFree(f.d_in);
        if (f.d_out) cudaFree(f.d_out);
        f.d_in = f.d_out = nullptr;
    }
    c->frame_w = c->frame_h = c->frame_pitch = 0;
}

void drop_batch_graphs(canny_ctx *c)
{
    drop_frame_graphs(c);
    for (auto &sl : c->slots)
        for (int v = 0; v < 2; ++v) {
            if (sl.exec[v]) cudaGraphExecDestroy(sl.exec[v]);
            if (sl.graph[v]) cudaGraphDestroy(sl.graph[v]);
            sl.exec[v] = nullptr;
            sl.graph[v] = nullptr;
            sl.valid[v] = false;
        }
}

void free_hyst(canny_ctx *c)
{
    drop_batch_graphs(c);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    if (c->hyst_mem) cudaFree(c->hyst_mem);
    c->hyst_mem = nullptr;
    c->hs = HystScratch{};
}

// (Re)allocate the hysteresis scratch for at least max_tiles tiles and max_imgs images.
canny_status ensure_hyst(canny_ctx *c, uint32_t max_tiles, uint32_t max_imgs)
{
    if (c->hyst_mem && c->hs.max_tiles >= max_tiles && c->hs.max_imgs >= max_imgs) return CANNY_OK;
    if (c->hyst_mem) {
        cudaDeviceSynchronize();
        max_tiles = max_tiles > c->hs.max_tiles ? max_tiles : c->hs.max_tiles;
        max_imgs = max_imgs > c->hs.max_imgs ? max_imgs : c->hs.max_imgs;
        free_hyst(c);
    }
    if (max_tiles < 1) max_tiles = 1;
    if (max_imgs < 1) max_imgs = 1;
    size_t off_imgs = 0;
    size_t off_masks = align_up(off_imgs + sizeof(HystImage) * max_imgs, 256);
    size_t off_pend = align_up(off_masks + sizeof(TileMasks) * max_tiles, 256);
    size_t off_stamp = align_up(off_pend + sizeof(uint32_t) * HT * (size_t)max_tiles, 256);
    size_t off_lists = align_up(off_stamp + sizeof(uint32_t) * (size_t)max_tiles, 256);
    size_t off_bits = align_up(off_lists + sizeof(uint32_t) * 2 * (size_t)max_tiles, 256);
    size_t off_uf_label = align_up(off_bits + sizeof(uint32_t) * 2 * HT * (size_t)max_tiles, 256);
    size_t off_uf_parent = align_up(off_uf_label + 128 * (size_t)max_tiles, 256);
    size_t off_uf_seeded = align_up(off_uf_parent + sizeof(uint32_t) * 64 * (size_t)max_tiles, 256);
    size_t off_queue = align_up(off_uf_seeded + 64 * (size_t)max_tiles, 256);
    size_t off_state = align_up(off_queue + sizeof(unsigned long long) * (size_t)max_tiles, 256);
    size_t total = align_up(off_state + sizeof(HystState), 256);
    void *mem = nullptr;
    cudaError_t e = dev_alloc(&mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CANNY_ENOMEM;
    }
    char *b = (char *)mem;
    c->hyst_mem = mem;
    c->hs.imgs = (HystImage *)(b + off_imgs);
    c->hs.masks = (TileMasks *)(b + off_masks);
    c->hs.pend_bits = (uint32_t *)(b + off_pend);
    c->hs.stamp = (uint32_t *)(b + off_stamp);
    c->hs.lists = (uint32_t *)(b + off_lists);
    c->hs.bits = (uint32_t *)(b + off_bits);
    c->hs.uf_label = (uint8_t *)(b + off_uf_label);
    c->hs.uf_parent = (uint32_t *)(b + off_uf_parent);
    c->hs.uf_seeded = (uint8_t *)(b + off_uf_seeded);
    c->hs.queue = (unsigned long long *)(b + off_queue);
    c->hs.state = (HystState *)(b + off_state);
    c->hs.max_tiles = max_tiles;
    c->hs.max_imgs = max_imgs;
    if (cudaMemset(c->hs.state, 0, sizeof(HystState)) != cudaSuccess) return CANNY_ECUDA;
    if (cudaMemset(c->hs.queue, 0, sizeof(unsigned long long) * max_tiles) != cudaSuccess) return CANNY_ECUDA;
    // (single images run their passes in one cooperative launch where the device
    // allows; the graph while-loop is the fallback)
    if (c->use_graph && !hyst_coop_supported()) {
        if (hyst_build_graph(c->hs, &c->graph, &c->exec) != cudaSuccess) {
            cudaGetLastError();
            c->use_graph = 0;
            c->graph = nullptr;
            c->exec = nullptr;
        }
    }
    return CANNY_OK;
}

uint32_t auto_max_passes(uint32_t ntiles)
{
    // Every pass that queues another promotes at least one pending border pixel
    // (at most 4 * 32 - 4 per tile), so this bound is never reached by a correct run.
    uint64_t cap = 64 + (uint64_t)(4 * HT - 4) * ntiles;
    return cap > 0x7fffffffu ? 0x7fffffffu : (uint32_t)cap;
}

// Queue the global passes of the current run (after hyst_reset + local fill).
canny_status run_global(canny_ctx *c, cudaStream_t s)
{
    // one cooperative launch runs every pass; else a graph while-loop; else the host loop
    if (c->use_graph && hyst_coop_supported() && !host_passes_injected()) {
        cudaError_t e = cudaSuccess;
        if (take_failure(g_fail_barrier)) e = launch_hyst_phantom_arrival(c->hs, s);   // test hook
        if (e == cudaSuccess) e = launch_hyst_global_coop(c->hs, s, (uint32_t)c->last.tiles);
        // a device shared with other work (fewer SMs than at start-up) may refuse
        // the grid: then the passes are driven from the host below
        if (e != cudaErrorCooperativeLaunchTooLarge) return from_cuda(e);
        cudaGetLastError();
    } else if (c->use_graph && c->exec) {
        return from_cuda(cudaGraphLaunch(c->exec, s));
    }
    // host-driven loop: one pass, read the control block, repeat
    for (;;) {
        cudaError_t e = launch_hyst_global_pass(c->hs, hyst_pass_grid(), false, 0, s);
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaMemcpyAsync(c->h_state, c->hs.state, sizeof(HystState), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
        const HystState *st = (const HystState *)c->h_state;
        if (!st->keep_going) return CANNY_OK;
    }
}

// per_dim: the image must fit max_w x max_h; otherwise only the pixel budget binds.
canny_status check_image(const canny_ctx *c, const canny_image *im, bool per_dim = true)
{
    if (!im) return CANNY_EINVAL;
    if (im->w < 0 || im->h < 0) return CANNY_EINVAL;
    if (im->w == 0 || im->h == 0) return CANNY_OK;
    if (per_dim && (im->w > c->max_w || im->h > c->max_h)) return CANNY_EINVAL;
    if ((int64_t)im->w * im->h > (int64_t)c->max_w * c->max_h) return CANNY_EINVAL;
    if (!im->d_in || !im->d_out) return CANNY_EINVAL;
    if (im->in_pitch < im->w || im->out_pitch < im->w) return CANNY_EINVAL;
    // the output must not overlap the input
    const char *a0 = (const char *)im->d_in, *a1 = a0 + (int64_t)(im->h - 1) * im->in_pitch + im->w;
    const char *b0 = (const char *)im->d_out, *b1 = b0 + (int64_t)(im->h - 1) * im->out_pitch + im->w;
    if (a0 < b1 && b0 < a1) return CANNY_EINVAL;
    return CANNY_OK;
}

int band_for(const canny_ctx *c, int w, int h);

// Steps 1-3 + thresholds into im->d_out as a class map.
canny_status run_stencil(canny_ctx *c, const canny_image *im, cudaStream_t s)
{
    if (c->p.path == CANNY_PATH_INT)
        return from_cuda(launch_k1_classify_u8(im->d_in, im->in_pitch, im->d_out, im->out_pitch,
                                               im->w, im->h, c->it, &c->hs.state->error, s,
                                               band_for(c, im->w, im->h)));
    if (!c->mag) {
        // the stored strength image is only needed for a class map of the float path
        if (dev_alloc((void **)&c->mag, sizeof(float) * (size_t)c->max_w * c->max_h) != cudaSuccess) {
            cudaGetLastError();
            return CANNY_ENOMEM;
        }
    }
    cudaError_t e = cudaMemsetAsync(c->d_max, 0, sizeof(float), s);
    if (e == cudaSuccess)
        e = launch_k1f_magnitude(im->d_in, im->in_pitch, c->mag, im->w, im->w, im->h, c->fp, true,
                                 c->d_max, s);
    if (e == cudaSuccess)
        e = launch_k1f_classify(c->mag, im->w, im->d_out, im->out_pitch, im->w, im->h, c->d_max,
                                c->fp.lo_frac, c->fp.hi_frac, s);
    return from_cuda(e);
}

HystImage hyst_image(const canny_image *im, uint32_t base)
{
    HystImage h = {};
    h.map = im->d_out;
    h.w = im->w;
    h.h = im->h;
    h.pitch = im->out_pitch;
    h.ntx = (im->w + HT - 1) / HT;
    h.nty = (im->h + HT - 1) / HT;
    h.tile_base = base;
    return h;
}

// A device buffer of at least need bytes (grown on demand; on growth, work still
// queued on the device may read the old buffer, so the device is drained first).
bool ensure_stage(uint8_t **buf, size_t *cap, size_t need)
{
    if (*cap >= need) return true;
    cudaDeviceSynchronize();
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (dev_alloc((void **)buf, need) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return false;
    }
    *cap = need;
    return true;
}

// An input the TMA path cannot read (base or pitch not 16-byte aligned) is
// copied into a 16-byte pitched staging buffer on the device first: the fused
// kernel's direct-load variant runs at about a third of the TMA variant's speed,
// the copy costs 2 bytes per pixel of HBM traffic. *im is updated to the copy.
canny_status stage_input(canny_ctx *c, canny_image *im, cudaStream_t s)
{
    if (c->direct_loads || tma_usable(im->d_in, im->in_pitch)) return CANNY_OK;
    const int pitch = (int)align_up((size_t)im->w, 16);
    if (!ensure_stage(&c->d_stage, &c->stage_cap, (size_t)pitch * im->h)) return CANNY_OK;   // direct loads
    const Repitch r = {im->d_in, c->d_stage, im->w, im->h, im->in_pitch, pitch};
    canny_status st = from_cuda(launch_repitch(r, s));
    if (st != CANNY_OK) return st;
    im->d_in = c->d_stage;
    im->in_pitch = pitch;
    return CANNY_OK;
}

// Float path, Steps 1-4 up to the tile-local hysteresis: pass 1 finds the largest
// squared strength, pass 2 recomputes the stencil and writes edges and tile state.
// The float path's strength and sector maps for a w x h image. Growing them
// drops the frame graphs, which hold the old buffer.
bool ensure_fmaps(canny_ctx *c, int w, int h)
{
    const size_t need = k1f_map_bytes(w, h);
    if (c->fmaps_cap >= need) return true;
    drop_frame_graphs(c);
    return ensure_stage(reinterpret_cast<uint8_t **>(&c->fmaps), &c->fmaps_cap, need);
}

// Float path, Steps 1-4 up to the tile-local hysteresis: pass 1 writes the
// squared strengths and sectors and finds their maximum, pass 2 suppresses,
// thresholds and fills the tiles from those maps.
canny_status run_float_fused(canny_ctx *c, const canny_image *im, const HystImage &himg, cudaStream_t s)
{
    if (!ensure_fmaps(c, im->w, im->h)) return CANNY_ENOMEM;
    cudaError_t e = cudaMemsetAsync(c->d_max, 0, sizeof(float), s);
    if (e == cudaSuccess)
        e = launch_k1f_strength(im->d_in, im->in_pitch, im->w, im->h, c->fp, c->d_max, c->fmaps, s);
    if (e == cudaSuccess) e = launch_k1f_nms(c->fmaps, im->w, im->h, c->fp, c->d_max, c->hs, himg, s);
    return from_cuda(e);
}

uint32_t max_passes_for(const canny_ctx *c, uint32_t ntiles)
{
    return c->p.max_passes > 0 ? (uint32_t)c->p.max_passes : auto_max_passes(ntiles);
}

// Chase budget of a single image's global passes (one cooperative launch, with
// the union-find stage after the first pass): the context's tuning, else 4
// tiles on the float path, else the kernels' own default (0). The float path's
// edge maps (smoothing at sigma 1.4, thresholds a fraction of the largest
// strength) hold long weak chains, and a short chase that leaves them to the
// union-find stage ends sooner than a long one (global stage at 16384^2: 0.106
// ms at 4 tiles, 0.141 at 16; at 4096^2: 0.073 against 0.108). Batches and
// frame sequences, whose one-launch-per-pass loop has no union-find stage,
// keep the default.
uint32_t chase_budget_of(const canny_ctx *c)
{
    if (c->chase_budget > 0) return (uint32_t)c->chase_budget;
    return c->p.path == CANNY_PATH_F32 ? 4u : 0u;
}

canny_status run_one(canny_ctx *c, const canny_image *im, cudaStream_t s, bool stencil = true)
{
    canny_status st = check_image(c, im);
    if (st != CANNY_OK) return st;
    c->last = canny_stats{};
    c->last.images = 1;
    c->last_stream = s;
    if (im->w == 0 || im->h == 0) return CANNY_OK;
    uint32_t ntiles = tiles_of(im->w, im->h);
    st = ensure_hyst(c, ntiles, 1);
    if (st != CANNY_OK) return st;
    c->last.pixels = (int64_t)im->w * im->h;
    c->last.tiles = ntiles;
    const int slot = (c->timing && c->ev_runs < (int)c->ev.size() / EV_PER_RUN) ? c->ev_runs++ : -1;
    cudaEvent_t *ev = slot >= 0 ? &c->ev[EV_PER_RUN * slot] : nullptr;
    if (ev) cudaEventRecord(ev[0], s);
    const HystImage himg = hyst_image(im, 0);
    st = from_cuda(hyst_reset(c->hs, ntiles, 1, max_passes_for(c, ntiles), s, &himg, chase_budget_of(c)));
    if (st != CANNY_OK) return st;
    if (ev) cudaEventRecord(ev[1], s);
    canny_image staged = *im;
    if (stencil) {
        st = stage_input(c, &staged, s);
        if (st != CANNY_OK) return st;
    }
    if (stencil && c->p.path == CANNY_PATH_INT) {
        // fused: Steps 1-3, thresholds and the tile-local fill in one kernel
        st = from_cuda(launch_k1_edges_u8(staged.d_in, staged.in_pitch, im->w, im->h, c->it, c->hs, himg, s,
                                          band_for(c, im->w, im->h)));
        if (st != CANNY_OK) return st;
        if (ev) {
            cudaEventRecord(ev[2], s);
            cudaEventRecord(ev[3], s);
        }
    } else if (stencil) {
        // float path: two stencil passes, the second fused with the tile-local fill
        st = run_float_fused(c, &staged, himg, s);
        if (st != CANNY_OK) return st;
        if (ev) {
            cudaEventRecord(ev[2], s);
            cudaEventRecord(ev[3], s);
        }
    } else {
        st = from_cuda(cudaMemcpy2DAsync(im->d_out, im->out_pitch, im->d_in, im->in_pitch, im->w, im->h,
                                         cudaMemcpyDeviceToDevice, s));
        if (st != CANNY_OK) return st;
        if (ev) cudaEventRecord(ev[2], s);
        st = from_cuda(launch_hyst_local_single(c->hs, himg, s));
        if (st != CANNY_OK) return st;
        if (ev) cudaEventRecord(ev[3], s);
    }
    st = run_global(c, s);
    if (ev) cudaEventRecord(ev[4], s);
    return st;
}

// ---------------------------------------------------------------- integer-path batches
// Blob layout, identical on host (pinned staging) and device: header, image
// descriptors, input tensor maps; the host copy also carries the HystImage
// array that is uploaded to the hysteresis scratch.
struct BlobLayout {
    size_t imgs, tmaps, stage, himgs, dev_bytes, host_bytes;
};

BlobLayout blob_layout(uint32_t cap)
{
    BlobLayout L;
    L.imgs = 128;
    L.tmaps = align_up(L.imgs + sizeof(BatchImage) * cap, 128);
    L.stage = align_up(L.tmaps + sizeof(CUtensorMap) * cap, 128);
    L.himgs = align_up(L.stage + sizeof(Repitch) * cap, 128);
    L.dev_bytes = L.himgs;
    L.host_bytes = L.himgs + sizeof(HystImage) * cap;
    return L;
}

canny_status ensure_blob(canny_ctx *c, uint32_t cap)
{
    if (c->d_blob && c->blob_cap >= cap) return CANNY_OK;
    cudaDeviceSynchronize();
    drop_batch_graphs(c);
    if (cap < 64) cap = 64;
    if (cap < c->blob_cap * 2) cap = c->blob_cap * 2;
    if (c->d_blob) cudaFree(c->d_blob);
    c->d_blob = nullptr;
    for (auto &sl : c->slots) {
        if (sl.h_blob) cudaFreeHost(sl.h_blob);
        sl.h_blob = nullptr;
    }
    c->blob_cap = 0;
    const BlobLayout L = blob_layout(cap);
    if (dev_alloc((void **)&c->d_blob, L.dev_bytes) != cudaSuccess) { cudaGetLastError(); return CANNY_ENOMEM; }
    for (auto &sl : c->slots) {
        if (pinned_alloc((void **)&sl.h_blob, L.host_bytes) != cudaSuccess) {
            cudaGetLastError();
            return CANNY_ENOMEM;
        }
        if (!sl.done && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) return CANNY_ECUDA;
    }
    c->blob_cap = cap;
    return CANNY_OK;
}

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    }
    return n;
}

// Band height of a single image's units: the configured one, else whichever of
// 32 and 64 rows needs fewer rows of work per SM slot (12 one-warp CTAs fit on
// an SM): max(units / slots, 1) waves x rows per unit. Images that do not fill
// the GPU twice over take the shorter units (measured: 7680 x 4320 0.163 against
// 0.176 ms, 512 x 512 0.109 against 0.144 ms; 16384^2 keeps 64 rows).
int band_for(const canny_ctx *c, int w, int h)
{
    if (c->band > 0) return c->band;
    const double slots = (double)sm_count() * 12.0;
    auto cost = [&](int band) {
        const double waves = (double)k1_units(w, h, band) / slots;
        return (waves > 1.0 ? waves : 1.0) * k1_band_rows(band);
    };
    return cost(32) < cost(64) ? 32 : 64;
}

// Band height of batch units: the configured one, else 64.
int batch_band(const canny_ctx *c) { return c->band > 0 ? c->band : 64; }

// The batch graph: upload descriptors -> reset, repitch inputs the TMA path
// cannot read -> fused kernel (persistent, pops units) -> while (work) global pass.
// Variant 1 holds the TMA-only fused kernel (every input TMA-readable).
canny_status build_batch_graph(canny_ctx *c, canny_ctx::Slot &sl, int v)
{
    if (sl.exec[v]) cudaGraphExecDestroy(sl.exec[v]);
    if (sl.graph[v]) cudaGraphDestroy(sl.graph[v]);
    sl.exec[v] = nullptr;
    sl.graph[v] = nullptr;
    sl.valid[v] = false;
    const BlobLayout L = blob_layout(c->blob_cap);
    BatchHeader *hdr = (BatchHeader *)c->d_blob;
    const BatchImage *imgs = (const BatchImage *)(c->d_blob + L.imgs);
    const CUtensorMap *tmaps = (const CUtensorMap *)(c->d_blob + L.tmaps);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return from_cuda(e);
    cudaGraphNode_t up1, up2, init, k1, loop;
    e = cudaGraphAddMemcpyNode1D(&up1, g, nullptr, 0, c->d_blob, sl.h_blob, L.dev_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaGraphAddMemcpyNode1D(&up2, g, nullptr, 0, c->hs.imgs, sl.h_blob + L.himgs,
                                     sizeof(HystImage) * c->blob_cap, cudaMemcpyHostToDevice);
    // (the worklist stamps need no clearing: the fused kernel writes every tile's stamp)
    if (e == cudaSuccess) e = hyst_add_init_from_header(g, &up1, 1, c->hs, hdr, &init);
    cudaGraphNode_t stage;
    if (e == cudaSuccess)
        e = add_repitch_list_node(g, &up1, 1, (const Repitch *)(c->d_blob + L.stage), hdr, &stage);
    cudaGraphNode_t d_k1[3] = {up2, init, stage};
    if (e == cudaSuccess)
        e = k1_add_batch_node(g, d_k1, 3, batch_band(c), v == 1, imgs, tmaps, hdr, c->it, c->hs,
                              c->ctas_per_sm > 0 ? sm_count() * c->ctas_per_sm : 0, &k1);
    sl.k1node[v] = k1;
    cudaGraphNode_t fill;
    if (e == cudaSuccess) e = hyst_add_fill(g, &k1, 1, c->hs, &fill);
    if (e == cudaSuccess && c->batch_passes == 1) {
        e = hyst_add_coop(g, &fill, 1, c->hs, &loop);
        if (e == cudaErrorNotSupported) {   // the device cannot hold the cooperative grid
            cudaGetLastError();
            e = hyst_add_loop(g, &fill, 1, c->hs, &loop);
        }
    } else if (e == cudaSuccess) {
        e = hyst_add_loop(g, &fill, 1, c->hs, &loop);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sl.exec[v], g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        sl.exec[v] = nullptr;
        return CANNY_ECUDA;
    }
    sl.graph[v] = g;
    sl.valid[v] = true;
    return CANNY_OK;
}

// Tensor map of an input image, encoded once per (pointer, size, pitch).
bool cached_map(canny_ctx *c, const canny_image *im, CUtensorMap *out)
{
    char key[96];
    snprintf(key, sizeof(key), "%p:%d:%d:%d", (const void *)im->d_in, im->w, im->h, im->in_pitch);
    auto it = c->tmaps.find(key);
    if (it != c->tmaps.end()) {
        *out = it->second;
        return true;
    }
    if (!encode_k1_map(out, im->d_in, im->w, im->h, im->in_pitch)) return false;
    if (c->tmaps.size() > 65536) c->tmaps.clear();
    c->tmaps.emplace(key, *out);
    return true;
}

canny_status run_batch_int(canny_ctx *c, int n, const canny_image *imgs, uint32_t nimg, uint32_t ntiles,
                           cudaStream_t s)
{
    canny_status st = ensure_blob(c, nimg);
    if (st != CANNY_OK) return st;
    // the graph uploads blob_cap image descriptors into the hysteresis scratch
    st = ensure_hyst(c, ntiles, c->blob_cap);
    if (st != CANNY_OK) return st;
    canny_ctx::Slot &sl = c->slots[c->next_slot];
    c->next_slot ^= 1;
    // the slot's staging buffer may still feed a batch launched two calls ago
    if (cudaEventSynchronize(sl.done) != cudaSuccess) return CANNY_ECUDA;
    const BlobLayout L = blob_layout(c->blob_cap);
    BatchHeader *hdr = (BatchHeader *)sl.h_blob;
    BatchImage *bi = (BatchImage *)(sl.h_blob + L.imgs);
    CUtensorMap *tm = (CUtensorMap *)(sl.h_blob + L.tmaps);
    Repitch *rp = (Repitch *)(sl.h_blob + L.stage);
    HystImage *hi = (HystImage *)(sl.h_blob + L.himgs);
    // inputs the TMA path cannot read are repitched into the batch staging
    // buffer by the graph's first kernel (direct loads run at about a third of
    // the TMA path's speed); if that buffer cannot be had they are read directly
    size_t stage_need = 0;
    for (int i = 0; i < n; ++i)
        if (imgs[i].w > 0 && imgs[i].h > 0 && !tma_usable(imgs[i].d_in, imgs[i].in_pitch))
            stage_need += align_up(align_up((size_t)imgs[i].w, 16) * (size_t)imgs[i].h, 256);
    const bool staged =
        !c->direct_loads && (stage_need == 0 || ensure_stage(&c->d_bstage, &c->bstage_cap, stage_need));
    uint32_t k = 0, tile_base = 0, unit_base = 0, nstage = 0, stage_tasks = 0;
    size_t stage_off = 0;
    bool all_tma = true;
    for (int i = 0; i < n; ++i) {
        canny_image im_use = imgs[i];
        const canny_image *im = &im_use;
        if (im->w == 0 || im->h == 0) continue;
        if (staged && !tma_usable(im->d_in, im->in_pitch)) {
            const int pitch = (int)align_up((size_t)im->w, 16);
            uint8_t *dst = c->d_bstage + stage_off;
            rp[nstage++] = Repitch{im->d_in, dst, im->w, im->h, im->in_pitch, pitch, stage_tasks};
            stage_tasks += repitch_tasks(im->w, im->h);
            stage_off += align_up((size_t)pitch * (size_t)im->h, 256);
            im_use.d_in = dst;
            im_use.in_pitch = pitch;
        }
        hi[k] = hyst_image(im, tile_base);
        BatchImage b = {};
        b.img = hi[k];
        b.in = im->d_in;
        b.in_pitch = im->in_pitch;
        b.unit_base = unit_base;
        b.nsx = (im->w + k1_strip_width() - 1) / k1_strip_width();
        b.tma = cached_map(c, im, &tm[k]) ? 1 : 0;
        all_tma = all_tma && b.tma;
        bi[k] = b;
        tile_base += tiles_of(im->w, im->h);
        unit_base += (uint32_t)k1_units(im->w, im->h, batch_band(c));
        ++k;
    }
    BatchHeader hh = {};
    hh.nimg = nimg;
    hh.total_units = unit_base;
    hh.next_unit = 0;
    hh.ntiles = ntiles;
    hh.max_passes = max_passes_for(c, ntiles);
    hh.nstage = nstage;
    hh.stage_tasks = stage_tasks;
    hh.chase_budget = (uint32_t)c->chase_budget;
    *hdr = hh;
    const int v = all_tma ? 1 : 0;
    if (!sl.valid[v]) {
        st = build_batch_graph(c, sl, v);
        if (st != CANNY_OK) return st;
    }
    cudaError_t e = cudaSuccess;
    if (c->ctas_per_sm <= 0)
        e = k1_set_batch_units(sl.exec[v], sl.k1node[v], batch_band(c), v == 1, (const BatchImage *)(c->d_blob + L.imgs),
                               (const CUtensorMap *)(c->d_blob + L.tmaps), (BatchHeader *)c->d_blob, c->it, c->hs,
                               unit_base);
    if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec[v], s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
    return from_cuda(e);
}

}  // namespace

namespace canny {

cudaError_t dev_alloc(void **p, size_t bytes)
{
    if (take_failure(g_fail_device)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void **p, size_t bytes)
{
    if (take_failure(g_fail_device)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}

bool arena_failure_injected() { return take_failure(g_fail_arena); }

bool host_passes_injected() { return take_failure(g_host_passes); }

canny_status batch_reserve(canny_ctx *c, uint32_t max_images, uint32_t max_tiles)
{
    if (!c || c->p.path != CANNY_PATH_INT) return CANNY_EINVAL;
    canny_status st = ensure_blob(c, max_images < 1 ? 1 : max_images);
    if (st == CANNY_OK) st = ensure_hyst(c, max_tiles, c->blob_cap);
    // the graphs for inputs the TMA path reads, instantiated now rather than
    // on a slot's first batch
    for (auto &sl : c->slots)
        if (st == CANNY_OK && !sl.valid[1]) st = build_batch_graph(c, sl, 1);
    return st;
}

}  // namespace canny

extern "C" {

canny_status canny_inject_faults(const canny_fault_injection *f)
{
    if (!f || f->device_allocations < 0 || f->arena_admissions < 0 || f->stalled_barriers < 0 ||
        f->host_driven_passes < 0)
        return CANNY_EINVAL;
    g_fail_device.store(f->device_allocations);
    g_fail_arena.store(f->arena_admissions);
    g_fail_barrier.store(f->stalled_barriers);
    g_host_passes.store(f->host_driven_passes);
    return CANNY_OK;
}

canny_status canny_params_default(canny_params *p)
{
    if (!p) return CANNY_EINVAL;
    p->path = CANNY_PATH_INT;
    p->sigma = 1.4f;
    p->ksize = 7;
    p->low = 40.f;
    p->high = 100.f;
    p->max_passes = 0;
    return CANNY_OK;
}

canny_status canny_create(int max_w, int max_h, const canny_params *p, canny_ctx **out)
{
    if (!out) return CANNY_EINVAL;
    *out = nullptr;
    if (max_w <= 0 || max_h <= 0) return CANNY_EINVAL;
    if ((int64_t)max_w * max_h > ((int64_t)1 << 34)) return CANNY_EINVAL;
    canny_status st = check_params(p);
    if (st != CANNY_OK) return st;

    canny_ctx *c = new (std::nothrow) canny_ctx();
    if (!c) return CANNY_ENOMEM;
    c->max_w = max_w;
    c->max_h = max_h;
    c->p = *p;
    if (p->path == CANNY_PATH_INT) {
        c->it.lo2 = (int)p->low * (int)p->low;
        c->it.hi2 = (int)p->high * (int)p->high;
    } else {
        // Step 1 taps: exp(-k^2 / (2 sigma^2)), normalised in double, rounded to float
        int r = p->ksize / 2;
        double g[MAX_KSIZE], sum = 0.0, sd = (double)p->sigma;
        for (int k = -r; k <= r; ++k) {
            g[k + r] = exp(-(double)(k * k) / (2.0 * sd * sd));
            sum += g[k + r];
        }
        for (int k = 0; k < p->ksize; ++k) c->fp.taps[k] = (float)(g[k] / sum);
        c->fp.ksize = p->ksize;
        c->fp.lo_frac = p->low;
        c->fp.hi_frac = p->high;
    }
    if (getenv("CANNY_NO_GRAPH")) c->use_graph = 0;

    cudaError_t e = pinned_alloc((void **)&c->h_state, sizeof(HystState));
    if (e != cudaSuccess) { cudaGetLastError(); delete c; return CANNY_ENOMEM; }
    e = cudaEventCreateWithFlags(&c->staging_free, cudaEventDisableTiming);
    if (e != cudaSuccess) { cudaGetLastError(); canny_destroy(c); return from_cuda(e); }
    st = ensure_hyst(c, tiles_of(max_w, max_h), 1);
    if (st != CANNY_OK) { canny_destroy(c); return st; }
    if (p->path == CANNY_PATH_F32) {
        e = dev_alloc((void **)&c->d_max, sizeof(float));
        if (e != cudaSuccess) { cudaGetLastError(); canny_destroy(c); return CANNY_ENOMEM; }
    }
    *out = c;
    return CANNY_OK;
}

void canny_destroy(canny_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_hyst(c);
    if (c->mag) cudaFree(c->mag);
    if (c->fmaps) cudaFree(c->fmaps);
    if (c->d_max) cudaFree(c->d_max);
    if (c->d_host_in) cudaFree(c->d_host_in);
    if (c->d_host_out) cudaFree(c->d_host_out);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->h_imgs) cudaFreeHost(c->h_imgs);
    if (c->staging_free) cudaEventDestroy(c->staging_free);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto &sl : c->slots) {
        if (sl.h_blob) cudaFreeHost(sl.h_blob);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (c->d_blob) cudaFree(c->d_blob);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_bstage) cudaFree(c->d_bstage);
    free_frames(c);
    for (auto &f : c->fslots) {
        if (f.up) cudaEventDestroy(f.up);
        if (f.comp) cudaEventDestroy(f.comp);
        if (f.down) cudaEventDestroy(f.down);
    }
    if (c->frame_start) cudaEventDestroy(c->frame_start);
    if (c->s_up) cudaStreamDestroy(c->s_up);
    if (c->s_down) cudaStreamDestroy(c->s_down);
    if (c->s_cap) cudaStreamDestroy(c->s_cap);
    if (c->d_frame_err) cudaFree(c->d_frame_err);
    delete c;
}

canny_status canny_run(canny_ctx *c, const uint8_t *d_in, uint8_t *d_out, void *stream)
{
    if (!c) return CANNY_EINVAL;
    canny_image im = {d_in, d_out, c->max_w, c->max_h, c->max_w, c->max_w};
    return run_one(c, &im, (cudaStream_t)stream);
}

canny_status canny_run_pitched(canny_ctx *c, const canny_image *img, void *stream)
{
    if (!c) return CANNY_EINVAL;
    return run_one(c, img, (cudaStream_t)stream);
}

canny_status canny_run_batch(canny_ctx *c, int n, const canny_image *imgs, void *stream)
{
    if (!c || n < 0 || (n > 0 && !imgs)) return CANNY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t pixels = 0;
    uint32_t ntiles = 0, nimg = 0;
    for (int i = 0; i < n; ++i) {
        canny_status st = check_image(c, &imgs[i], false);
        if (st != CANNY_OK) return st;
        pixels += (int64_t)imgs[i].w * imgs[i].h;
        uint32_t t = tiles_of(imgs[i].w, imgs[i].h);
        if (t) { ntiles += t; ++nimg; }
    }
    if (pixels > (int64_t)c->max_w * c->max_h) return CANNY_EINVAL;
    c->last = canny_stats{};
    c->last.images = n;
    c->last.pixels = pixels;
    c->last.tiles = ntiles;
    c->last_stream = s;
    if (nimg == 0) return CANNY_OK;
    if (c->p.path == CANNY_PATH_INT) return run_batch_int(c, n, imgs, nimg, ntiles, s);
    canny_status st = ensure_hyst(c, ntiles, nimg);
    if (st != CANNY_OK) return st;
    if (c->h_imgs_cap < nimg) {
        cudaEventSynchronize(c->staging_free);
        if (c->h_imgs) cudaFreeHost(c->h_imgs);
        c->h_imgs = nullptr;
        c->h_imgs_cap = 0;
        if (pinned_alloc((void **)&c->h_imgs, sizeof(HystImage) * nimg) != cudaSuccess) {
            cudaGetLastError();
            return CANNY_ENOMEM;
        }
        c->h_imgs_cap = nimg;
    }
    // the staging buffer may still feed the previous batch's upload
    cudaError_t e = cudaEventSynchronize(c->staging_free);
    if (e != cudaSuccess) return from_cuda(e);
    uint32_t base = 0, k = 0;
    for (int i = 0; i < n; ++i) {
        uint32_t t = tiles_of(imgs[i].w, imgs[i].h);
        if (!t) continue;
        c->h_imgs[k++] = hyst_image(&imgs[i], base);
        base += t;
    }
    e = cudaMemcpyAsync(c->hs.imgs, c->h_imgs, sizeof(HystImage) * nimg, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(c->staging_free, s);
    if (e != cudaSuccess) return from_cuda(e);
    st = from_cuda(hyst_reset(c->hs, ntiles, nimg, max_passes_for(c, ntiles), s, nullptr, (uint32_t)c->chase_budget));
    if (st != CANNY_OK) return st;
    base = 0;
    for (int i = 0; i < n; ++i) {
        const uint32_t t = tiles_of(imgs[i].w, imgs[i].h);
        if (!t) continue;
        st = run_float_fused(c, &imgs[i], hyst_image(&imgs[i], base), s);
        if (st != CANNY_OK) return st;
        base += t;
    }
    return run_global(c, s);
}

canny_status canny_run_host(canny_ctx *c, const uint8_t *h_in, int in_pitch, uint8_t *h_out,
                            int out_pitch, int w, int h, void *stream)
{
    if (!c || !h_in || !h_out || w < 0 || h < 0 || w > c->max_w || h > c->max_h) return CANNY_EINVAL;
    if (in_pitch < w || out_pitch < w) return CANNY_EINVAL;
    if (w == 0 || h == 0) return CANNY_OK;
    cudaStream_t s = (cudaStream_t)stream;
    size_t cap = (size_t)c->max_w * c->max_h;
    if (!c->d_host_in) {
        if (dev_alloc((void **)&c->d_host_in, cap) != cudaSuccess ||
            dev_alloc((void **)&c->d_host_out, cap) != cudaSuccess) {
            cudaGetLastError();
            return CANNY_ENOMEM;
        }
    }
    cudaError_t e = cudaMemcpy2DAsync(c->d_host_in, w, h_in, in_pitch, w, h, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return from_cuda(e);
    canny_image im = {c->d_host_in, c->d_host_out, w, h, w, w};
    canny_status st = run_one(c, &im, s);
    if (st != CANNY_OK) return st;
    e = cudaMemcpy2DAsync(h_out, out_pitch, c->d_host_out, w, w, h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_state, c->hs.state, sizeof(HystState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    const HystState *hst = (const HystState *)c->h_state;
    return (hst->error & 10u) ? CANNY_ECUDA : (hst->error & 1u) ? CANNY_ENOCONVERGE : CANNY_OK;
}

canny_status canny_hysteresis(canny_ctx *c, const canny_image *img, void *stream)
{
    if (!c) return CANNY_EINVAL;
    return run_one(c, img, (cudaStream_t)stream, false);
}

canny_status canny_classify(canny_ctx *c, const canny_image *img, void *stream)
{
    if (!c) return CANNY_EINVAL;
    canny_status st = check_image(c, img);
    if (st != CANNY_OK) return st;
    if (img->w == 0 || img->h == 0) return CANNY_OK;
    return run_stencil(c, img, (cudaStream_t)stream);
}

canny_status canny_magnitude_f32(canny_ctx *c, const canny_image *img, float *d_mag, int d_mag_pitch,
                                 float *d_max, void *stream)
{
    if (!c || !img || !d_mag || !d_max) return CANNY_EINVAL;
    if (c->p.path != CANNY_PATH_F32) return CANNY_EUNSUPPORTED;
    if (img->w < 0 || img->h < 0 || img->w > c->max_w || img->h > c->max_h) return CANNY_EINVAL;
    if (img->w == 0 || img->h == 0) return CANNY_OK;
    if (!img->d_in || img->in_pitch < img->w || d_mag_pitch < img->w) return CANNY_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // the production float kernel's own strengths: pass 1 into the context's maps,
    // then M = sqrt_rn(s) per pixel
    if (!ensure_fmaps(c, img->w, img->h)) return CANNY_ENOMEM;
    cudaError_t e = cudaMemsetAsync(c->d_max, 0, sizeof(float), s);
    if (e == cudaSuccess)
        e = launch_k1f_strength(img->d_in, img->in_pitch, img->w, img->h, c->fp, c->d_max, c->fmaps, s);
    if (e == cudaSuccess)
        e = launch_k1f_strength_out(c->fmaps, img->w, img->h, d_mag, d_mag_pitch, c->d_max, d_max, s);
    return from_cuda(e);
}

canny_status canny_enable_timing(canny_ctx *c, int enable)
{
    if (!c) return CANNY_EINVAL;
    if (enable && c->ev.empty()) {
        c->ev.resize(EV_PER_RUN * 4096, nullptr);
        for (auto &e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return CANNY_ECUDA; }
    }
    c->timing = enable ? 1 : 0;
    c->ev_runs = 0;
    return CANNY_OK;
}

canny_status canny_read_timing(canny_ctx *c, canny_timing *out)
{
    if (!c || !out) return CANNY_EINVAL;
    *out = canny_timing{};
    for (int r = 0; r < c->ev_runs; ++r) {
        cudaEvent_t *e = &c->ev[EV_PER_RUN * r];
        if (cudaEventSynchronize(e[4]) != cudaSuccess) { c->ev_runs = 0; return CANNY_ECUDA; }
        float z = 0, a = 0, b = 0, g = 0, t = 0;
        cudaEventElapsedTime(&z, e[0], e[1]);
        cudaEventElapsedTime(&a, e[1], e[2]);
        cudaEventElapsedTime(&b, e[2], e[3]);
        cudaEventElapsedTime(&g, e[3], e[4]);
        cudaEventElapsedTime(&t, e[0], e[4]);
        out->reset_ms += z;
        out->stencil_ms += a;
        out->local_ms += b;
        out->global_ms += g;
        out->total_ms += t;
        out->runs += 1;
    }
    c->ev_runs = 0;
    return CANNY_OK;
}

canny_status canny_set_tuning(canny_ctx *c, const canny_tuning *t)
{
    if (!c || !t) return CANNY_EINVAL;
    if ((t->band != 0 && !k1_band_supported(t->band)) || t->ctas_per_sm < 0 || t->ctas_per_sm > 32)
        return CANNY_EINVAL;
    if (t->direct_loads != 0 && t->direct_loads != 1) return CANNY_EINVAL;
    if (t->chase_budget < 0 || t->chase_budget > 4096) return CANNY_EINVAL;
    if (t->batch_passes != 0 && t->batch_passes != 1) return CANNY_EINVAL;
    c->direct_loads = t->direct_loads;
    // frame graphs hold the chase budget of their reset node; batch graphs hold the rest
    if (t->band != c->band || t->ctas_per_sm != c->ctas_per_sm || t->batch_passes != c->batch_passes ||
        t->chase_budget != c->chase_budget) {
        cudaDeviceSynchronize();
        drop_batch_graphs(c);
        c->band = t->band;
        c->ctas_per_sm = t->ctas_per_sm;
        c->batch_passes = t->batch_passes;
        c->chase_budget = t->chase_budget;
    }
    return CANNY_OK;
}

canny_status canny_get_tuning(const canny_ctx *c, canny_tuning *out)
{
    if (!c || !out) return CANNY_EINVAL;
    *out = canny_tuning{};
    out->band = c->band;
    out->ctas_per_sm = c->ctas_per_sm;
    out->direct_loads = c->direct_loads;
    out->chase_budget = c->chase_budget;
    out->batch_passes = c->batch_passes;
    return CANNY_OK;
}

canny_status canny_autotune_batch(canny_ctx *c, int n, const canny_image *imgs, void *stream,
                                  const char *cache_path, canny_tuning *out)
{
    if (!c || n < 0 || (n > 0 && !imgs)) return CANNY_EINVAL;
    if (c->p.path != CANNY_PATH_INT) return CANNY_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    // size class of the batch: image count and mean image area, in octaves
    int64_t px = 0;
    int nimg = 0;
    bool unaligned = false;
    for (int i = 0; i < n; ++i) {
        if (imgs[i].w > 0 && imgs[i].h > 0) {
            px += (int64_t)imgs[i].w * imgs[i].h;
            ++nimg;
            unaligned = unaligned || !tma_usable(imgs[i].d_in, imgs[i].in_pitch);
        }
    }
    if (nimg == 0) return CANNY_EINVAL;
    int dev = 0;
    cudaDeviceProp prop;
    cudaGetDevice(&dev);
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CANNY_ECUDA;
    char key[320];   // device name (at most 256) + the size classes
    snprintf(key, sizeof(key), "%s|int|n%d|a%d|u%d|v2", prop.name, (int)log2((double)nimg),
             (int)log2((double)px / nimg), unaligned ? 1 : 0);
    canny_tuning best = {};
    best.direct_loads = c->direct_loads;
    if (cache_path && *cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[640];
            while (fgets(line, sizeof(line), f)) {
                char k[320];
                canny_tuning t = {};
                if (sscanf(line,
                           "{\"key\": \"%319[^\"]\", \"band\": %d, \"ctas_per_sm\": %d, \"direct_loads\": %d, "
                           "\"chase_budget\": %d, \"batch_passes\": %d, \"ms\": %lf}",
                           k, &t.band, &t.ctas_per_sm, &t.direct_loads, &t.chase_budget, &t.batch_passes,
                           &t.ms) == 7 &&
                    strcmp(k, key) == 0) {
                    best = t;
                    best.from_cache = 1;
                }
            }
            fclose(f);
        }
    }
    if (!best.from_cache) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return CANNY_ECUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return CANNY_ECUDA;
        }
        // one candidate: a warm-up run, then two timed runs; best is replaced if faster
        auto trial = [&](canny_tuning cand) -> canny_status {
            canny_status st = canny_set_tuning(c, &cand);
            if (st == CANNY_OK) st = canny_run_batch(c, n, imgs, stream);
            if (st == CANNY_OK && cudaEventRecord(e0, s) != cudaSuccess) st = CANNY_ECUDA;
            for (int r = 0; r < 2 && st == CANNY_OK; ++r) st = canny_run_batch(c, n, imgs, stream);
            if (st == CANNY_OK && cudaEventRecord(e1, s) != cudaSuccess) st = CANNY_ECUDA;
            if (st == CANNY_OK && cudaEventSynchronize(e1) != cudaSuccess) st = CANNY_ECUDA;
            if (st != CANNY_OK) return st;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 2 < best.ms) {
                best = cand;
                best.ms = ms / 2;
            }
            return CANNY_OK;
        };
        canny_status st = CANNY_OK;
        best.ms = 1e30;
        // stage 1, tile shape: rows per unit x persistent CTAs per SM
        const int bands[3] = {32, 64, 160};
        const int ctas[3] = {0, 12, 16};
        const canny_tuning base = best;
        for (int bi = 0; bi < 3 && st == CANNY_OK; ++bi)
            for (int ci = 0; ci < 3 && st == CANNY_OK; ++ci) {
                canny_tuning cand = base;
                cand.band = bands[bi];
                cand.ctas_per_sm = ctas[ci];
                st = trial(cand);
            }
        // stage 2, halo layout of inputs the TMA path cannot read: repitched or direct loads
        if (unaligned && st == CANNY_OK) {
            canny_tuning cand = best;
            cand.direct_loads = 1 - best.direct_loads;
            st = trial(cand);
        }
        // stage 3, pass schedule: chase budget x while-loop or one cooperative node
        const int budgets[3] = {4, 16, 64};
        const canny_tuning shape = best;
        for (int bi = 0; bi < 3 && st == CANNY_OK; ++bi)
            for (int p = 0; p < 2 && st == CANNY_OK; ++p) {
                canny_tuning cand = shape;
                cand.chase_budget = budgets[bi];
                cand.batch_passes = p;
                if (cand.chase_budget == 16 && p == 0 && shape.chase_budget == 0 && shape.batch_passes == 0)
                    continue;   // the defaults, timed in stage 1
                st = trial(cand);
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != CANNY_OK) return st;
        best.from_cache = 0;
        if (cache_path && *cache_path) {
            FILE *f = fopen(cache_path, "a");
            if (f) {
                fprintf(f,
                        "{\"key\": \"%s\", \"band\": %d, \"ctas_per_sm\": %d, \"direct_loads\": %d, "
                        "\"chase_budget\": %d, \"batch_passes\": %d, \"ms\": %.6f}\n",
                        key, best.band, best.ctas_per_sm, best.direct_loads, best.chase_budget, best.batch_passes,
                        best.ms);
                fclose(f);
            }
        }
    }
    canny_status st = canny_set_tuning(c, &best);
    if (st != CANNY_OK) return st;
    if (out) *out = best;
    return CANNY_OK;
}

// ---------------------------------------------------------------- frame sequences
namespace {

// Streams, events and the error word, created once.
canny_status ensure_frame_streams(canny_ctx *c)
{
    if (c->s_up) return CANNY_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_down, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->frame_start, cudaEventDisableTiming);
    for (auto &f : c->fslots) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.up, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.comp, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.down, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = dev_alloc((void **)&c->d_frame_err, sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    return CANNY_OK;
}

// One frame's pipeline on slot f as a graph: { reset -> stencil (+ tile fill) }
// captured as a child graph, then the global-pass while-loop, then the error OR.
canny_status build_frame_graph(canny_ctx *c, canny_ctx::FrameSlot &f)
{
    const canny_image im = {f.d_in, f.d_out, c->frame_w, c->frame_h, c->frame_pitch, c->frame_pitch};
    const uint32_t ntiles = tiles_of(im.w, im.h);
    const HystImage himg = hyst_image(&im, 0);
    cudaGraph_t body = nullptr, g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->s_cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return from_cuda(e);
    canny_status st = from_cuda(hyst_reset(c->hs, ntiles, 1, max_passes_for(c, ntiles), c->s_cap, &himg,
                                           (uint32_t)c->chase_budget));
    if (st == CANNY_OK) {
        if (c->p.path == CANNY_PATH_INT)
            st = from_cuda(launch_k1_edges_u8(im.d_in, im.in_pitch, im.w, im.h, c->it, c->hs, himg, c->s_cap,
                                              band_for(c, im.w, im.h)));
        else
            st = run_float_fused(c, &im, himg, c->s_cap);
    }
    e = cudaStreamEndCapture(c->s_cap, &body);
    if (st == CANNY_OK && e != cudaSuccess) st = from_cuda(e);
    if (st != CANNY_OK) {
        cudaGetLastError();
        if (body) cudaGraphDestroy(body);
        return st;
    }
    cudaGraphNode_t child, loop, eor;
    e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, g, nullptr, 0, body);
    if (e == cudaSuccess) e = hyst_add_loop(g, &child, 1, c->hs, &loop);
    if (e == cudaSuccess) e = hyst_add_error_or(g, &loop, 1, c->hs, c->d_frame_err, &eor);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&f.exec, g, 0);
    cudaGraphDestroy(body);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        f.exec = nullptr;
        return from_cuda(e);
    }
    f.graph = g;
    return CANNY_OK;
}

canny_status ensure_frames(canny_ctx *c, int w, int h)
{
    canny_status st = ensure_frame_streams(c);
    if (st != CANNY_OK) return st;
    const int pitch = (w + 15) / 16 * 16;                 // 16-byte rows: the TMA path
    const size_t need = (size_t)pitch * (size_t)h;
    if ((size_t)c->frame_pitch * (size_t)c->frame_h < need || !c->fslots[0].d_in) {
        free_frames(c);
        for (auto &f : c->fslots) {
            if (dev_alloc((void **)&f.d_in, need) != cudaSuccess || dev_alloc((void **)&f.d_out, need) != cudaSuccess) {
                cudaGetLastError();
                free_frames(c);
                return CANNY_ENOMEM;
            }
        }
    } else if (c->frame_w != w || c->frame_h != h) {
        drop_frame_graphs(c);
    }
    c->frame_w = w;
    c->frame_h = h;
    c->frame_pitch = pitch;
    // the float path's maps exist before any frame graph captures their address
    if (c->p.path != CANNY_PATH_INT && !ensure_fmaps(c, w, h)) return CANNY_ENOMEM;
    for (auto &f : c->fslots) {
        if (f.exec) continue;
        st = build_frame_graph(c, f);
        if (st != CANNY_OK) return st;
    }
    return CANNY_OK;
}

}  // namespace

canny_status canny_run_frames(canny_ctx *c, int n, const uint8_t *const *h_in, int in_pitch,
                              uint8_t *const *h_out, int out_pitch, int w, int h, void *stream)
{
    if (!c || n < 0 || w < 0 || h < 0 || w > c->max_w || h > c->max_h) return CANNY_EINVAL;
    if (n > 0 && (!h_in || !h_out)) return CANNY_EINVAL;
    if (n == 0 || w == 0 || h == 0) return CANNY_OK;
    if (in_pitch < w || out_pitch < w) return CANNY_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!h_in[i] || !h_out[i]) return CANNY_EINVAL;
    const uint32_t ntiles = tiles_of(w, h);
    canny_status st = ensure_hyst(c, ntiles, 1);
    if (st != CANNY_OK) return st;
    st = ensure_frames(c, w, h);
    if (st != CANNY_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int pitch = c->frame_pitch;
    cudaError_t e = cudaMemsetAsync(c->d_frame_err, 0, sizeof(uint32_t), s);
    // the copy streams start after everything already queued on s
    if (e == cudaSuccess) e = cudaEventRecord(c->frame_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_up, c->frame_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_down, c->frame_start, 0);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        canny_ctx::FrameSlot &f = c->fslots[i & 1];
        // upload frame i once the pipeline of frame i-2 has read this slot's input
        if (i >= 2) e = cudaStreamWaitEvent(c->s_up, f.comp, 0);
        if (e == cudaSuccess)
            e = (in_pitch == w && pitch == w)   // contiguous: one linear copy
                    ? cudaMemcpyAsync(f.d_in, h_in[i], (size_t)w * h, cudaMemcpyHostToDevice, c->s_up)
                    : cudaMemcpy2DAsync(f.d_in, pitch, h_in[i], in_pitch, w, h, cudaMemcpyHostToDevice, c->s_up);
        if (e == cudaSuccess) e = cudaEventRecord(f.up, c->s_up);
        // pipeline of frame i once it is uploaded and frame i-2's edges are downloaded
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, f.up, 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(s, f.down, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(f.exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(f.comp, s);
        // download frame i's edges
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_down, f.comp, 0);
        if (e == cudaSuccess)
            e = (out_pitch == w && pitch == w)
                    ? cudaMemcpyAsync(h_out[i], f.d_out, (size_t)w * h, cudaMemcpyDeviceToHost, c->s_down)
                    : cudaMemcpy2DAsync(h_out[i], out_pitch, f.d_out, pitch, w, h, cudaMemcpyDeviceToHost, c->s_down);
        if (e == cudaSuccess) e = cudaEventRecord(f.down, c->s_down);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->fslots[(n - 1) & 1].down, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_state, c->d_frame_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    c->last = canny_stats{};
    c->last.images = n;
    c->last.pixels = (int64_t)n * w * h;
    c->last.tiles = ntiles;
    c->last_stream = s;
    const uint32_t err = c->h_state[0];
    return (err & 10u) ? CANNY_ECUDA : (err & 1u) ? CANNY_ENOCONVERGE : CANNY_OK;
}

canny_status canny_get_stats(canny_ctx *c, canny_stats *out)
{
    if (!c || !out) return CANNY_EINVAL;
    *out = c->last;
    if (c->last.tiles == 0) { out->status = CANNY_OK; return CANNY_OK; }
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->h_state, c->hs.state, sizeof(HystState), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        out->status = from_cuda(e);
        return (canny_status)out->status;
    }
    const HystState *st = (const HystState *)c->h_state;
    out->hyst_passes = st->pass;
    out->hyst_tiles_visited = st->visited;
    out->pending_tiles = st->pending_tiles;
    out->status = (st->error & 10u) ? CANNY_ECUDA : (st->error & 1u) ? CANNY_ENOCONVERGE : CANNY_OK;
    return CANNY_OK;
}

const char *canny_strerror(canny_status s)
{
    switch (s) {
    case CANNY_OK: return "ok";
    case CANNY_EINVAL: return "invalid argument";
    case CANNY_ENOMEM: return "out of memory";
    case CANNY_ECUDA: return "CUDA error";
    case CANNY_ENOCONVERGE: return "hysteresis did not converge within the pass cap";
    case CANNY_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

}  // extern "C"
