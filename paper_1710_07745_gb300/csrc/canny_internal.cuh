// canny_internal.cuh -- types shared by the kernels and the C ABI of libcanny.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "canny.h"

namespace canny {

// ---------------------------------------------------------------- hysteresis tiles
// Hysteresis (Step 4 of the paper's Sec. 2.2.1) works on 32x32 pixel tiles: one
// warp per tile, one lane per row, one 32-bit mask per row.
constexpr int HT = 32;

// One image as the hysteresis kernels see it: its edge map (written in place)
// and where its tiles start in the global tile numbering.
struct HystImage {
    uint8_t *map;       // edge map (device), h rows of pitch bytes
    int w, h, pitch;
    int ntx, nty;       // tiles across and down
    uint32_t tile_base; // global index of the image's tile (0, 0)
    uint32_t pad;
};

// Per-tile border masks, written by the local fill and updated by global passes.
// edge_*: which border pixels are edges; pend_*: which border pixels are weak
// pixels not (yet) connected to an edge. Bit i of top/bottom is column i, bit i
// of left/right is row i.
struct TileMasks {
    uint32_t edge_top, edge_bottom, edge_left, edge_right;
    uint32_t pend_top, pend_bottom, pend_left, pend_right;
};

// Device-side control block of one run's hysteresis.
// Checked builds (-DCANNY_CHECKS, in place of a sanitizer): device-side bounds
// checks that record a failure in the run's error word (bit 3) and skip the
// access. In normal builds a check is the constant true and compiles away.
#ifdef CANNY_CHECKS
#define CANNY_CHECK(cond, errp) ((cond) ? true : (atomicOr((errp), 8u), false))
#else
#define CANNY_CHECK(cond, errp) true
#endif

// Nanoseconds of the GPU's global timer: bounds the waits of device-side spins by
// time, not by an iteration count whose duration depends on the clock and load.
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr uint64_t WAIT_TIMEOUT_NS = 1000000000ull;   // a device-side wait gives up after a second

struct HystState {
    uint32_t list_count[2];   // sizes of the two worklists
    uint32_t done_ctas;       // CTAs finished in the current global pass
    uint32_t pass;            // global passes completed
    uint32_t max_passes;      // cap
    uint32_t error;           // bit 0: cap reached with work left; bit 1: a pipeline wait ran out;
                              // bit 3: a bounds check of a checked build failed
    uint32_t visited;         // tile visits summed over passes
    uint32_t pending_tiles;   // tiles with unresolved weak pixels after the local fill
    uint32_t ntiles;          // tiles in this run
    uint32_t nimg;            // images in this run
    uint32_t keep_going;      // 1 if another pass is needed
    uint32_t bar_count, bar_gen;   // grid barrier of the cooperative multi-pass kernel
    uint32_t uf_entries;      // union-find stage: entries of the pass before it (list of that pass)
    uint32_t uf_count;        // union-find stage: tiles listed (in list 1)
    uint32_t chase_budget;    // tiles a chain may be followed into within a pass (0: the default)
    // the in-pass queue of a global pass (zero between passes)
    uint32_t q_head, q_tail;  // queue slots claimed by consumers / reserved by producers
    uint32_t q_open;          // queued items not yet finished, plus CTAs still on their worklist entries
    uint32_t q_waiters;       // warps that stay for queued items
    uint32_t run_tag;         // 1..65535, new for every run: tags queue items of this run
};

struct HystScratch {
    HystImage *imgs;          // [max_imgs]
    TileMasks *masks;         // [max_tiles]
    uint32_t *pend_bits;      // [max_tiles * 32]: weak-not-edge pixels, one word per tile row
    uint32_t *bits;           // [max_tiles * 64]: the stencil's class bits per tile, rows 0..31
                              // of class >= 1 (weak or strong), then rows 0..31 of class 2
    uint32_t *stamp;          // [max_tiles]: last pass a tile was queued for
    uint32_t *lists;          // [2 * max_tiles]
    HystState *state;
    uint32_t max_tiles;
    uint32_t max_imgs;
    // union-find over the border components of pending pixels (the global passes'
    // stage for long chains; null: passes only)
    uint8_t *uf_label;        // [max_tiles * 128]: component of each of the 124 border pixels, count at 127
    uint32_t *uf_parent;      // [max_tiles * 64]: parent of component 64 t + j
    uint8_t *uf_seeded;       // [max_tiles * 64]: component touches an edge of a neighbouring tile
    // in-pass queue of the global passes: (run tag << 48) | (budget << 32) | tile,
    // 0 when empty; zeroed once at allocation, each slot re-zeroed by its consumer
    unsigned long long *queue;   // [max_tiles]
};

// ---------------------------------------------------------------- stencil launch data
// Integer-path thresholds, squared.
struct IntThresholds {
    int lo2, hi2;
};

constexpr int MAX_KSIZE = 31;
struct FloatParams {
    float taps[MAX_KSIZE];
    int ksize;
    float lo_frac, hi_frac;
};

// ---------------------------------------------------------------- batches
// One image of a batch as the fused kernel sees it.
struct BatchImage {
    HystImage img;             // output map and tile geometry
    const uint8_t *in;
    int in_pitch;
    uint32_t unit_base;        // index of the image's first (strip, band) unit
    int nsx;                   // strips across
    int tma;                   // 1 if tmaps[k] describes the input
    int pad[2];
};

// Device header of a batch run, uploaded with the descriptors.
struct BatchHeader {
    uint32_t nimg, total_units, next_unit, ntiles, max_passes;
    uint32_t nstage, stage_tasks;   // inputs repitched into staging first (Repitch list), their tasks
    uint32_t chase_budget;          // the global passes' chase budget (0: the default)
};

// ---------------------------------------------------------------- launchers (k1_fused.cu)
// Band heights the fused kernel is built for (rows per unit of work).
bool k1_band_supported(int band);
// Input rows a unit of the given band height processes (its band plus halos).
int k1_band_rows(int band);
int k1_units(int w, int h, int band);
int k1_strip_width();
bool encode_k1_map(void *tmap_out, const uint8_t *in, int w, int h, int in_pitch);
// Integer Steps 1-3 + thresholds: class map (0/1/2) into cls. err: device word
// that gets bit 1 if a shared-memory pipeline wait ran out.
cudaError_t launch_k1_classify_u8(const uint8_t *in, int in_pitch, uint8_t *cls, int cls_pitch,
                                  int w, int h, IntThresholds t, uint32_t *err, cudaStream_t s, int band = 64);
// Integer Steps 1-4 up to the tile-local hysteresis: edges (0/255) into img.map,
// tile masks / pending bitmaps / first worklist into hs (after hyst_reset).
cudaError_t launch_k1_edges_u8(const uint8_t *in, int in_pitch, int w, int h, IntThresholds t,
                               const HystScratch &hs, HystImage img, cudaStream_t s, int band = 64);
// The same for every image of a batch, as a node of graph g: with ctas > 0 a
// persistent grid of `ctas` one-warp CTAs pops (image, strip, band) units from
// hdr->next_unit; with ctas <= 0 the grid has one CTA per unit, set before each
// launch of the instantiated graph by k1_set_batch_units.
// tma_only: every image's input is TMA-readable (the kernel holds no direct-load path).
cudaError_t k1_add_batch_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, int band, bool tma_only,
                              const BatchImage *imgs, const CUtensorMap *tmaps, BatchHeader *hdr, IntThresholds t,
                              const HystScratch &hs, int ctas, cudaGraphNode_t *out);
cudaError_t k1_set_batch_units(cudaGraphExec_t exec, cudaGraphNode_t node, int band, bool tma_only,
                               const BatchImage *imgs, const CUtensorMap *tmaps, BatchHeader *hdr, IntThresholds t,
                               const HystScratch &hs, uint32_t units);

// ---------------------------------------------------------------- host images (hostio.cu)
// One image between a tight, 16-byte aligned, device-accessible host buffer and
// a pitched device buffer.
struct HostCopy {
    uint8_t *host;       // gather: source; scatter: destination (h rows of w bytes, no padding)
    uint8_t *dev;        // gather: destination; scatter: source (h rows of dev_pitch bytes)
    int w, h, dev_pitch, pad;
};
// True if host (pitch bytes per row, w wide) can take the kernel path: pinned and
// mapped at the same address, 16-byte aligned, rows without padding.
bool host_copy_ok(const void *host, int pitch, int w);
uint64_t host_copy_words(int w, int h);
// Copies d_copies[0 .. n) (a device array, n <= 65535) in one launch; total_words =
// the sum of host_copy_words over the copies.
cudaError_t launch_gather(const HostCopy *d_copies, int n, uint64_t total_words, cudaStream_t s);
cudaError_t launch_scatter(const HostCopy *d_copies, int n, uint64_t total_words, cudaStream_t s);
// A device image (any pitch and alignment) copied into 16-byte pitched rows.
struct Repitch {
    const uint8_t *src;
    uint8_t *dst;        // 16-byte aligned, dst_pitch a multiple of 16
    int w, h, src_pitch, dst_pitch;
    uint32_t task_base;  // in a list: tasks of the copies before this one
};
cudaError_t launch_repitch(const Repitch &c, cudaStream_t s);
// Graph node copying list[0 .. hdr->nstage) (read when the node runs; tasks
// counted by repitch_tasks, hdr->stage_tasks in all).
uint32_t repitch_tasks(int w, int h);
cudaError_t add_repitch_list_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const Repitch *list,
                                  const BatchHeader *hdr, cudaGraphNode_t *out);

// ---------------------------------------------------------------- allocation (canny_api.cu)
// Every device and pinned-host allocation of the library goes through these, so
// that canny_inject_faults can make the next ones fail (host side only).
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t pinned_alloc(void **p, size_t bytes);
// True (and one injected failure used up) if the serving arena's next request
// allocation is to fail.
bool arena_failure_injected();

// ---------------------------------------------------------------- TMA (tma.cu)
bool tma_usable(const void *base, int pitch);
bool encode_u8_map(void *tmap_out, const void *base, int w, int h, int pitch, int box_w, int box_h);

// ---------------------------------------------------------------- launchers (k1_stencil_f32.cu)
cudaError_t launch_k1f_magnitude(const uint8_t *in, int in_pitch, float *mag, int mag_pitch,
                                 int w, int h, const FloatParams &fp, bool nms, float *d_max,
                                 cudaStream_t s);
cudaError_t launch_k1f_classify(const float *mag_nms, int mag_pitch, uint8_t *cls, int cls_pitch,
                                int w, int h, const float *d_max, float lo_frac, float hi_frac,
                                cudaStream_t s);

// ---------------------------------------------------------------- launchers (k1_fused_f32.cu)
// Bytes of the float path's maps for a w x h image (squared strengths and
// gradient sectors of whole 64 x 128 blocks).
size_t k1f_map_bytes(int w, int h);
// Float path pass 1: Steps 1-2 and the sector of Step 3 into maps (k1f_map_bytes
// bytes, 16-byte aligned); the image's largest squared strength atomicMax'ed
// into *d_smax (as float bits; the caller zeroes it first).
cudaError_t launch_k1f_strength(const uint8_t *in, int in_pitch, int w, int h, const FloatParams &fp,
                                float *d_smax, void *maps, cudaStream_t s);
// The strengths of pass 1's maps: M = sqrt_rn(s) per pixel into mag (mag_pitch
// floats a row), Mmax = sqrt_rn(*d_smax) into *d_max.
cudaError_t launch_k1f_strength_out(const void *maps, int w, int h, float *mag, int mag_pitch, const float *d_smax,
                                    float *d_max, cudaStream_t s);
// Float path pass 2: Step 3 and the thresholds relative to sqrt(*d_smax) from the
// maps, then the tile-local hysteresis: edges into img.map, tile state into hs
// (after hyst_reset).
cudaError_t launch_k1f_nms(const void *maps, int w, int h, const FloatParams &fp, const float *d_smax,
                           const HystScratch &hs, HystImage img, cudaStream_t s);

// ---------------------------------------------------------------- launchers (hysteresis.cu)
// Tile fill from the fused stencil's class bits (hs.bits): grows every tile's
// strong pixels through its weak ones, writes 255/0 into img.map and the tile
// state the global passes read (after hyst_reset).
cudaError_t launch_hyst_fill_single(const HystScratch &hs, HystImage img, cudaStream_t s);
// The same over every tile of a batch, as a graph node (tile count and images read
// from the control block and hs.imgs when it runs).
cudaError_t hyst_add_fill(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out);
// Local fill over all tiles of one image whose class map is already in img.map.
cudaError_t launch_hyst_local_single(const HystScratch &hs, HystImage img, cudaStream_t s);
// Local fill over all tiles of the images already uploaded to hs.imgs.
cudaError_t launch_hyst_local_batch(const HystScratch &hs, uint32_t ntiles, uint32_t nimg,
                                    cudaStream_t s);
// One global pass over the current worklist. graph_cond: conditional handle to set
// (0 when not in a graph).
cudaError_t launch_hyst_global_pass(const HystScratch &hs, int grid, bool in_graph,
                                    unsigned long long cond_handle, cudaStream_t s);
// Every global pass in one cooperative launch (passes separated by a bounded
// grid barrier): cudaErrorNotSupported when the device cannot hold the grid.
bool hyst_coop_supported();
// Test hook (canny_inject_faults): true, and one count used up, if the next
// single-image global passes are to be driven from the host as when the device
// refuses the cooperative grid.
bool host_passes_injected();
// Integer-path batches: size the context's descriptor blob and hysteresis
// scratch for batches of up to max_images images and max_tiles tiles, so that
// no later batch of that size grows them (a growth synchronises the device and
// rebuilds the batch graphs), and instantiate the batch graphs.
canny_status batch_reserve(canny_ctx *c, uint32_t max_images, uint32_t max_tiles);
// All global passes of a single image in one cooperative launch: a grid of
// 2 x SMs CTAs, or fewer for an image of ntiles tiles (0: the full grid).
cudaError_t launch_hyst_global_coop(const HystScratch &hs, cudaStream_t s, uint32_t ntiles = 0);
// Test hook: barrier arrivals that no CTA makes, so the next cooperative
// launch's barrier never completes and its bounded wait runs out.
cudaError_t launch_hyst_phantom_arrival(const HystScratch &hs, cudaStream_t s);
// Clear the worklist stamps and the control block before a run; for a single
// image, also store its descriptor as image 0 (the global passes read it).
cudaError_t hyst_reset(const HystScratch &hs, uint32_t ntiles, uint32_t nimg,
                       uint32_t max_passes, cudaStream_t s, const HystImage *single = nullptr,
                       uint32_t chase_budget = 0);
int hyst_pass_grid();
// Executable graph { while (cond) global pass } bound to this scratch.
cudaError_t hyst_build_graph(const HystScratch &hs, cudaGraph_t *graph_out, cudaGraphExec_t *exec_out);
// Graph pieces for the batch graph.
cudaError_t hyst_add_loop(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out);
// Every global pass as one cooperative kernel node (long chains resolved by the
// union-find stage); cudaErrorNotSupported where the device cannot hold the grid.
cudaError_t hyst_add_coop(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out);
// Append { *acc |= state->error } after the given nodes (errors of one run of a
// sequence survive the next run's reset).
cudaError_t hyst_add_error_or(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                              uint32_t *acc, cudaGraphNode_t *out);
cudaError_t hyst_add_init_from_header(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps,
                                      const HystScratch &hs, const BatchHeader *hdr, cudaGraphNode_t *out);

}  // namespace canny
