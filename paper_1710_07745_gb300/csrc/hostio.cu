// hostio.cu -- moving images into (and out of) 16-byte pitched device buffers:
// tight host buffers, many in one launch, and device inputs whose base or pitch
// the TMA path cannot use. The copy engines move a pitched (2D) copy row by row,
// which for request-sized images (rows of about a kilobyte) runs at a fraction
// of the host link's rate; these kernels instead read (or write) the tight host
// image as one contiguous range of aligned 16-byte words over the link, and
// place the bytes into (or take them from) the pitched device rows. The host
// buffers must be device-accessible (pinned) and 16-byte aligned; the caller
// checks.
#include "canny_internal.cuh"

namespace canny {

namespace {

constexpr int IO_THREADS = 256;

// The 16 bytes at p, any alignment, from a source whose bytes are [lo, hi):
// two aligned 16-byte loads funnel-shifted into place, byte loads only where
// an aligned granule would reach outside [lo, hi) (bytes at or past hi read 0).
// The gather and the repitching below write whole aligned 16-byte destination
// words from it: destination word j of a copy is 16 bytes at row j / wpr,
// column 16 (j % wpr), wpr = ceil(w / 16); the bytes past w in a row's last
// word are don't-care padding.
__device__ __forceinline__ uint4 span16(const uint8_t *p, const uint8_t *lo, const uint8_t *hi)
{
    const uintptr_t pa = (uintptr_t)p, ga = pa & ~(uintptr_t)15, l = (uintptr_t)lo, h = (uintptr_t)hi;
    const int m = (int)(pa - ga);
    if (m == 0 && pa + 16 <= h) return __ldg(reinterpret_cast<const uint4 *>(p));
    if (m != 0 && ga >= l && ga + 32 <= h) {
        const uint4 A = __ldg(reinterpret_cast<const uint4 *>(ga));
        const uint4 B = __ldg(reinterpret_cast<const uint4 *>(ga + 16));
        const int q = m >> 2, r = 8 * (m & 3);
        // V[i] = word q + i of the 32 loaded bytes
        const uint32_t v0 = q == 0 ? A.x : q == 1 ? A.y : q == 2 ? A.z : A.w;
        const uint32_t v1 = q == 0 ? A.y : q == 1 ? A.z : q == 2 ? A.w : B.x;
        const uint32_t v2 = q == 0 ? A.z : q == 1 ? A.w : q == 2 ? B.x : B.y;
        const uint32_t v3 = q == 0 ? A.w : q == 1 ? B.x : q == 2 ? B.y : B.z;
        const uint32_t v4 = q == 0 ? B.x : q == 1 ? B.y : q == 2 ? B.z : B.w;
        return make_uint4(__funnelshift_r(v0, v1, r), __funnelshift_r(v1, v2, r), __funnelshift_r(v2, v3, r),
                          __funnelshift_r(v3, v4, r));
    }
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (pa + k < h) wd[k >> 2] |= (uint32_t)__ldg(p + k) << (8 * (k & 3));
    return make_uint4(wd[0], wd[1], wd[2], wd[3]);
}

// One copy per blockIdx.y; the CTAs of that row of the grid stride over its
// 16-byte words.

// host (tight rows) -> device (pitched rows): each thread writes one 16-byte
// word of a destination row (16-byte aligned rows; the bytes past w in a row's
// last word are don't-care padding) from the 16 source bytes at its offset in
// the tight image (span16: aligned 16-byte host loads funnel-shifted into
// place, byte loads at the image's ends).
__global__ void __launch_bounds__(IO_THREADS)
gather_kernel(const HostCopy *__restrict__ copies)
{
    const HostCopy c = copies[blockIdx.y];
    const uint64_t bytes = (uint64_t)c.w * (uint64_t)c.h;
    const uint32_t wpr = (uint32_t)(c.w + 15) >> 4;
    const uint64_t words = (uint64_t)wpr * (uint64_t)c.h;
    const bool aligned = ((((uintptr_t)c.dev) | (uintptr_t)c.dev_pitch) & 15) == 0;
    for (uint64_t j = blockIdx.x * (uint64_t)IO_THREADS + threadIdx.x; j < words; j += (uint64_t)gridDim.x * IO_THREADS) {
        const uint32_t y = (uint32_t)(j / wpr), x = 16u * (uint32_t)(j - (uint64_t)y * wpr);
        const uint64_t o = (uint64_t)y * (uint64_t)c.w + x;
        const uint4 v = span16(c.host + o, c.host, c.host + bytes);
        uint8_t *dst = c.dev + (int64_t)y * c.dev_pitch + x;
        if (aligned) {
            *reinterpret_cast<uint4 *>(dst) = v;
        } else {
            const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
            const int n = min(16, c.w - (int)x);
            for (int k = 0; k < n; ++k) dst[k] = (uint8_t)(wd[k >> 2] >> (8 * (k & 3)));
        }
    }
}

// device (pitched rows) -> host (tight rows)
__global__ void __launch_bounds__(IO_THREADS)
scatter_kernel(const HostCopy *__restrict__ copies)
{
    const HostCopy c = copies[blockIdx.y];
    const uint64_t bytes = (uint64_t)c.w * (uint64_t)c.h, words = (bytes + 15) / 16;
    for (uint64_t word = blockIdx.x * (uint64_t)IO_THREADS + threadIdx.x; word < words;
         word += (uint64_t)gridDim.x * IO_THREADS) {
        const uint64_t first = word * 16u;
        uint8_t b[16];
        int row = (int)(first / (uint64_t)c.w), col = (int)(first - (uint64_t)row * c.w);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            b[k] = first + k < bytes ? c.dev[(int64_t)row * c.dev_pitch + col] : 0;
            if (++col == c.w) {
                col = 0;
                ++row;
            }
        }
        if (first + 16 <= bytes) {
            uint32_t wd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                wd[q] = (uint32_t)b[4 * q] | ((uint32_t)b[4 * q + 1] << 8) | ((uint32_t)b[4 * q + 2] << 16) |
                        ((uint32_t)b[4 * q + 3] << 24);
            *reinterpret_cast<uint4 *>(c.host + first) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (first + k < bytes) c.host[first + k] = b[k];
        }
    }
}

int sm_total()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    }
    return sms;
}

// CTAs per copy: about eight resident CTAs per SM over the whole launch.
dim3 io_grid(int n, uint64_t total_words)
{
    const int sms = sm_total();
    const uint64_t per_copy = total_words / (uint64_t)n;                  // average words per copy
    uint64_t x = (uint64_t)sms * 8 / (uint64_t)n;
    const uint64_t useful = (per_copy + IO_THREADS - 1) / IO_THREADS;       // CTAs one copy can keep busy
    if (x > useful) x = useful;
    if (x < 1) x = 1;
    return dim3((unsigned)x, (unsigned)n);
}

__device__ __forceinline__ void repitch_word(const Repitch &c, uint64_t j)
{
    const uint32_t wpr = (uint32_t)(c.w + 15) >> 4;
    const uint32_t y = (uint32_t)(j / wpr), x = 16u * (uint32_t)(j - (uint64_t)y * wpr);
    const uint8_t *hi = c.src + (int64_t)(c.h - 1) * c.src_pitch + c.w;
    const uint4 v = span16(c.src + (int64_t)y * c.src_pitch + x, c.src, hi);
    *reinterpret_cast<uint4 *>(c.dst + (int64_t)y * c.dst_pitch + x) = v;
}

__host__ __device__ __forceinline__ uint64_t repitch_words(int w, int h) { return (uint64_t)((w + 15) / 16) * (uint64_t)h; }

__global__ void __launch_bounds__(IO_THREADS)
repitch_kernel(Repitch c)
{
    const uint64_t total = repitch_words(c.w, c.h);
    for (uint64_t j = blockIdx.x * (uint64_t)IO_THREADS + threadIdx.x; j < total; j += (uint64_t)gridDim.x * IO_THREADS)
        repitch_word(c, j);
}

// A list of copies: task t is destination words [64 t', 64 t' + 64) of the copy
// whose tasks hold t (t' = t - task_base). Each warp takes a contiguous range of
// tasks, finds its first copy by binary search and walks forward from there.
constexpr uint32_t TASK_WORDS = 64;

__global__ void __launch_bounds__(IO_THREADS)
repitch_list_kernel(const Repitch *__restrict__ list, const BatchHeader *__restrict__ hdr)
{
    const uint32_t n = hdr->nstage, T = hdr->stage_tasks;
    if (n == 0 || T == 0) return;
    const uint32_t wpc = IO_THREADS / 32, warps = gridDim.x * wpc, gw = blockIdx.x * wpc + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t t = (uint32_t)((uint64_t)T * gw / warps);
    const uint32_t tend = (uint32_t)((uint64_t)T * (gw + 1) / warps);
    if (t >= tend) return;
    int lo = 0, hi = (int)n - 1;                    // last copy whose tasks start at or before t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (list[mid].task_base <= t) lo = mid;
        else hi = mid - 1;
    }
    Repitch c = list[lo];
    uint32_t next = lo + 1 < (int)n ? list[lo + 1].task_base : T;
    for (; t < tend; ++t) {
        while (t >= next) {
            ++lo;
            c = list[lo];
            next = lo + 1 < (int)n ? list[lo + 1].task_base : T;
        }
        const uint64_t words = repitch_words(c.w, c.h);
        const uint64_t j0 = (uint64_t)(t - c.task_base) * TASK_WORDS + lane;
        if (j0 < words) repitch_word(c, j0);
        if (j0 + 32 < words) repitch_word(c, j0 + 32);
    }
}

}  // namespace

cudaError_t launch_repitch(const Repitch &c, cudaStream_t s)
{
    if (c.w <= 0 || c.h <= 0) return cudaSuccess;
    if ((((uintptr_t)c.dst) | (uintptr_t)c.dst_pitch) & 15) return cudaErrorInvalidValue;
    const uint64_t need = (repitch_words(c.w, c.h) + IO_THREADS - 1) / IO_THREADS, cap = (uint64_t)sm_total() * 8;
    repitch_kernel<<<(unsigned)(need < cap ? need : cap), IO_THREADS, 0, s>>>(c);
    return cudaGetLastError();
}

uint32_t repitch_tasks(int w, int h)
{
    return (uint32_t)((repitch_words(w, h) + TASK_WORDS - 1) / TASK_WORDS);
}

cudaError_t add_repitch_list_node(cudaGraph_t g, const cudaGraphNode_t *deps, size_t ndeps, const Repitch *list,
                                  const BatchHeader *hdr, cudaGraphNode_t *out)
{
    void *args[] = {(void *)&list, (void *)&hdr};
    cudaKernelNodeParams kp = {};
    kp.func = (void *)repitch_list_kernel;
    kp.gridDim = dim3((unsigned)sm_total() * 8);
    kp.blockDim = dim3(IO_THREADS);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(out, g, deps, ndeps, &kp);
}

bool host_copy_ok(const void *host, int pitch, int w)
{
    if (!host || pitch != w || (((uintptr_t)host) & 15) != 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // pinned host memory visible to the device at the same address (unified addressing)
    return a.type == cudaMemoryTypeHost && a.devicePointer == host;
}

uint64_t host_copy_words(int w, int h) { return ((uint64_t)w * (uint64_t)h + 15) / 16; }

cudaError_t launch_gather(const HostCopy *d_copies, int n, uint64_t total_words, cudaStream_t s)
{
    if (n <= 0 || total_words == 0) return cudaSuccess;
    if (n > 65535) return cudaErrorInvalidValue;
    gather_kernel<<<io_grid(n, total_words), IO_THREADS, 0, s>>>(d_copies);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const HostCopy *d_copies, int n, uint64_t total_words, cudaStream_t s)
{
    if (n <= 0 || total_words == 0) return cudaSuccess;
    if (n > 65535) return cudaErrorInvalidValue;
    scatter_kernel<<<io_grid(n, total_words), IO_THREADS, 0, s>>>(d_copies);
    return cudaGetLastError();
}

}  // namespace canny
