// noalloc.cu -- canny_run_noalloc: the integer pipeline for callers that cannot
// allocate device memory. The hysteresis scratch (tile masks, pending bitmaps,
// worklists, control block) lives in one fixed file-scope device array instead
// of context memory, so the call needs no context and allocates nothing.
#include <mutex>

#include "canny_internal.cuh"

namespace canny {
namespace {

// Largest image: 16384 tiles of 32x32 pixels (16.8 Mpixel, e.g. 4096 x 4096);
// the scratch holds per tile its masks, pending bitmap, stamp, worklist slots,
// in-pass queue slot and the stencil's class bits (436 bytes), about 7 MB in all.
constexpr uint32_t NOALLOC_MAX_TILES = 16384;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_IMGS = 0;
constexpr size_t OFF_MASKS = align256(OFF_IMGS + sizeof(HystImage));
constexpr size_t OFF_PEND = align256(OFF_MASKS + sizeof(TileMasks) * NOALLOC_MAX_TILES);
constexpr size_t OFF_STAMP = align256(OFF_PEND + sizeof(uint32_t) * HT * NOALLOC_MAX_TILES);
constexpr size_t OFF_LISTS = align256(OFF_STAMP + sizeof(uint32_t) * NOALLOC_MAX_TILES);
constexpr size_t OFF_BITS = align256(OFF_LISTS + sizeof(uint32_t) * 2 * NOALLOC_MAX_TILES);
constexpr size_t OFF_QUEUE = align256(OFF_BITS + sizeof(uint32_t) * 2 * HT * NOALLOC_MAX_TILES);
constexpr size_t OFF_STATE = align256(OFF_QUEUE + sizeof(unsigned long long) * NOALLOC_MAX_TILES);
constexpr size_t SCRATCH_BYTES = align256(OFF_STATE + sizeof(HystState));   // about 7 MB

// Shared by every call on a device; every device that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the array on the current device, looked up once per device.
// In host code g_noalloc_scratch is only a host-side stand-in for the symbol.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

canny_status status_of(cudaError_t e)
{
    return e == cudaSuccess ? CANNY_OK : CANNY_ECUDA;
}

}  // namespace
}  // namespace canny

using namespace canny;

extern "C" canny_status canny_run_noalloc(const uint8_t *d_in, int in_pitch, uint8_t *d_out,
                                          int out_pitch, int w, int h, int low, int high,
                                          void *stream)
{
    if (w < 0 || h < 0) return CANNY_EINVAL;
    if (w == 0 || h == 0) return CANNY_OK;
    if (!d_in || !d_out || in_pitch < w || out_pitch < w) return CANNY_EINVAL;
    if (low < 0 || high < low || high >= 32768) return CANNY_EINVAL;
    const char *a0 = (const char *)d_in, *a1 = a0 + (int64_t)(h - 1) * in_pitch + w;
    const char *b0 = (const char *)d_out, *b1 = b0 + (int64_t)(h - 1) * out_pitch + w;
    if (a0 < b1 && b0 < a1) return CANNY_EINVAL;
    const uint64_t ntiles = (uint64_t)((w + HT - 1) / HT) * (uint64_t)((h + HT - 1) / HT);
    if (ntiles > NOALLOC_MAX_TILES) return CANNY_EUNSUPPORTED;

    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return CANNY_ECUDA;
    char *b = (char *)base;
    HystScratch hs = {};
    hs.imgs = (HystImage *)(b + OFF_IMGS);
    hs.masks = (TileMasks *)(b + OFF_MASKS);
    hs.pend_bits = (uint32_t *)(b + OFF_PEND);
    hs.stamp = (uint32_t *)(b + OFF_STAMP);
    hs.lists = (uint32_t *)(b + OFF_LISTS);
    hs.bits = (uint32_t *)(b + OFF_BITS);
    hs.queue = (unsigned long long *)(b + OFF_QUEUE);   // zero-initialised with the array
    hs.state = (HystState *)(b + OFF_STATE);
    hs.max_tiles = NOALLOC_MAX_TILES;
    hs.max_imgs = 1;

    cudaStream_t s = (cudaStream_t)stream;
    IntThresholds t = {low * low, high * high};
    HystImage im = {};
    im.map = d_out;
    im.w = w;
    im.h = h;
    im.pitch = out_pitch;
    im.ntx = (w + HT - 1) / HT;
    im.nty = (h + HT - 1) / HT;
    im.tile_base = 0;
    // hyst_reset clears the control block; the tile fill rewrites the pending
    // bitmaps, masks and queue stamp of every tile of this image, and the fused
    // stencil its class bits, so a previous call's leftovers are never read
    const uint32_t cap = (uint32_t)(64 + (uint64_t)(4 * HT - 4) * ntiles);
    e = hyst_reset(hs, (uint32_t)ntiles, 1, cap, s, &im);
    if (e != cudaSuccess) return status_of(e);
    e = launch_k1_edges_u8(d_in, in_pitch, w, h, t, hs, im, s);
    if (e != cudaSuccess) return status_of(e);
    // global passes: one cooperative launch runs them all where the device allows;
    // if it refuses the grid (a device shared with other work), the host drives
    // them: one pass, read the control block, repeat
    HystState st = {};
    if (hyst_coop_supported() && !host_passes_injected()) {
        e = launch_hyst_global_coop(hs, s, (uint32_t)ntiles);
        if (e != cudaErrorCooperativeLaunchTooLarge) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(&st, hs.state, sizeof(st), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return status_of(e);
            return (st.error & 10u) ? CANNY_ECUDA : (st.error & 1u) ? CANNY_ENOCONVERGE : CANNY_OK;
        }
        cudaGetLastError();   // the refusal is not left pending for the caller's next CUDA call
    }
    for (;;) {
        e = launch_hyst_global_pass(hs, hyst_pass_grid(), false, 0, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&st, hs.state, sizeof(st), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return status_of(e);
        if (!st.keep_going) break;
    }
    return (st.error & 10u) ? CANNY_ECUDA : (st.error & 1u) ? CANNY_ENOCONVERGE : CANNY_OK;
}
