// tile_fill.cu -- the tile-local part of Step 4 of the paper's Sec. 2.2.1
// (hysteresis) for the integer path: the fused stencil leaves, per 32 x 32 tile,
// the rows of pixels of class >= 1 and of class 2 (2 bits a pixel); this kernel
// grows every tile's strong pixels through its weak ones, writes the tile's
// 255/0 edge bytes, and leaves the tile border masks, pending bitmaps and the
// first worklist for the global passes (hysteresis.cu).
#include "hyst_tile.cuh"

namespace canny {

namespace {

using namespace tile;

// Four tiles per warp (lane 8 tt + sl holds rows 4 sl .. 4 sl + 3 of tile 4 w + tt),
// from the fused stencil's per-tile class bits. A single image passes its
// descriptor and tile count; a batch reads them from hs.imgs and the control
// block (a graph node, fixed grid, grid-stride loop).
constexpr int FILL_WARPS = 8;
constexpr int FILL_THREADS = FILL_WARPS * 32;

template <bool SINGLE>
__global__ void __launch_bounds__(FILL_THREADS, 6)
hyst_fill_kernel(HystScratch hs, HystImage single, uint32_t ntiles_single)
{
    __shared__ uint32_t s_queued, s_pending, s_base;
    const int lane = threadIdx.x & 31, tt = lane >> 3, sl = lane & 7, warp = threadIdx.x >> 5;
    const uint32_t ntiles = SINGLE ? ntiles_single : hs.state->ntiles;
    const int nimg = SINGLE ? 1 : (int)hs.state->nimg;
    // a block-uniform loop: 4 FILL_WARPS tiles per CTA per step
    for (uint32_t b0 = blockIdx.x * 4u * FILL_WARPS; b0 < ntiles; b0 += gridDim.x * 4u * FILL_WARPS) {
        if (threadIdx.x == 0) s_queued = s_pending = 0u;
        __syncthreads();
        const uint32_t t = b0 + 4u * warp + (uint32_t)tt;
        const bool valid = t < ntiles && CANNY_CHECK(t < hs.max_tiles, &hs.state->error);
        HystImage im = single;
        int tx = 0, ty = 0;
        uint32_t c[4] = {0u, 0u, 0u, 0u}, e[4] = {0u, 0u, 0u, 0u};
        if (valid) {
            if (!SINGLE) im = hs.imgs[find_image(hs.imgs, nimg, t)];
            const uint32_t local = t - im.tile_base;
            tx = (int)(local % (uint32_t)im.ntx);
            ty = (int)(local / (uint32_t)im.ntx);
            const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(hs.bits + (size_t)t * 2 * HT + 4 * sl));
            const uint4 b = __ldcs(reinterpret_cast<const uint4 *>(hs.bits + (size_t)t * 2 * HT + HT + 4 * sl));
            c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
            e[0] = b.x; e[1] = b.y; e[2] = b.z; e[3] = b.w;
        }
        const uint32_t f = finish4(hs, im, tx, ty, t, valid, c, e, lane);
        // the CTA's queued tiles take consecutive worklist slots: one global atomic per CTA
        uint32_t rank = 0u;
        if (f & 1u) rank = atomicAdd(&s_queued, 1u);
        if (f & 2u) atomicAdd(&s_pending, 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base = s_queued ? atomicAdd(&hs.state->list_count[0], s_queued) : 0u;
            if (s_pending) atomicAdd(&hs.state->pending_tiles, s_pending);
        }
        __syncthreads();
        if (f & 1u) {
            const uint32_t i = s_base + rank;
            if (CANNY_CHECK(i < hs.max_tiles, &hs.state->error)) hs.lists[i] = t;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_hyst_fill_single(const HystScratch &hs, HystImage img, cudaStream_t s)
{
    const uint32_t ntiles = (uint32_t)img.ntx * (uint32_t)img.nty;
    if (ntiles == 0) return cudaSuccess;
    const int grid = (int)((ntiles + 4 * FILL_WARPS - 1) / (4 * FILL_WARPS));
    hyst_fill_kernel<true><<<grid, FILL_THREADS, 0, s>>>(hs, img, ntiles);
    return cudaGetLastError();
}

// Append the tile fill of a batch: a grid of SMs x 8 CTAs walks every tile.
cudaError_t hyst_add_fill(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const HystScratch &hs,
                          cudaGraphNode_t *out)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    HystScratch h = hs;
    HystImage none = {};
    uint32_t zero = 0;
    void *args[] = {&h, &none, &zero};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)hyst_fill_kernel<false>;
    kp.gridDim = dim3((unsigned)sms * 8u);
    kp.blockDim = dim3(FILL_THREADS);
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

}  // namespace canny
