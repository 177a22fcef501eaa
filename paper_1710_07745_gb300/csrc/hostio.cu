// hostio.cu -- moving images into (and out of) 16-byte pitched device buffers:
// tight host buffers, many in one launch, and device inputs whose base or pitch
// the TMA path cannot use. The copy engines move a pitched (2D) copy row by row,
// which for request-sized images (rows of about a kilobyte) runs at a fraction
// of the host link's rate; these kernels instead read (or write) the tight host
// image as one contiguous range of 16-byte words over the link, and place the
// bytes into (or take them from) the pitched device rows. The host buffers must
// be device-accessible (pinned) and 16-byte aligned; the caller checks.
#include "canny_internal.cuh"

namespace canny {

namespace {

constexpr int IO_THREADS = 256;

// One copy per blockIdx.y; the CTAs of that row of the grid stride over its
// 16-byte words of the tight host image.

// host (tight rows) -> device (pitched rows)
__global__ void __launch_bounds__(IO_THREADS)
gather_kernel(const HostCopy *__restrict__ copies)
{
    const HostCopy c = copies[blockIdx.y];
    const uint64_t bytes = (uint64_t)c.w * (uint64_t)c.h, words = (bytes + 15) / 16;
    for (uint64_t word = blockIdx.x * (uint64_t)IO_THREADS + threadIdx.x; word < words;
         word += (uint64_t)gridDim.x * IO_THREADS) {
        const uint64_t first = word * 16u;
        uint8_t b[16];
        if (first + 16 <= bytes) {
            const uint4 v = *reinterpret_cast<const uint4 *>(c.host + first);
            const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 16; ++k) b[k] = (uint8_t)(wd[k >> 2] >> (8 * (k & 3)));
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) b[k] = first + k < bytes ? c.host[first + k] : 0;
        }
        int row = (int)(first / (uint64_t)c.w), col = (int)(first - (uint64_t)row * c.w);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (first + k < bytes) c.dev[(int64_t)row * c.dev_pitch + col] = b[k];
            if (++col == c.w) {
                col = 0;
                ++row;
            }
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

// One 16-byte chunk of a destination row (chunk i of copy c): byte loads from
// the source (served by L1), one 16-byte store.
__device__ __forceinline__ void repitch_chunk(const Repitch &c, uint64_t i)
{
    const int chunks = (c.w + 15) / 16;
    const int y = (int)(i / (uint64_t)chunks), x = 16 * (int)(i - (uint64_t)y * chunks);
    const uint8_t *src = c.src + (int64_t)y * c.src_pitch + x;
    const int n = min(16, c.w - x);
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < 16; ++k)
        if (k < n) wd[k >> 2] |= (uint32_t)__ldg(src + k) << (8 * (k & 3));
    uint8_t *dst = c.dst + (int64_t)y * c.dst_pitch + x;
    if (n == 16) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < n) dst[k] = (uint8_t)(wd[k >> 2] >> (8 * (k & 3)));
    }
}

__global__ void __launch_bounds__(IO_THREADS)
repitch_kernel(Repitch c)
{
    const uint64_t total = (uint64_t)((c.w + 15) / 16) * (uint64_t)c.h;
    for (uint64_t i = blockIdx.x * (uint64_t)IO_THREADS + threadIdx.x; i < total; i += (uint64_t)gridDim.x * IO_THREADS)
        repitch_chunk(c, i);
}

}  // namespace

cudaError_t launch_repitch(const Repitch &c, cudaStream_t s)
{
    if (c.w <= 0 || c.h <= 0) return cudaSuccess;
    if ((((uintptr_t)c.dst) | (uintptr_t)c.dst_pitch) & 15) return cudaErrorInvalidValue;
    const uint64_t work = (uint64_t)((c.w + 15) / 16) * (uint64_t)c.h;
    const uint64_t need = (work + IO_THREADS - 1) / IO_THREADS, cap = (uint64_t)sm_total() * 8;
    repitch_kernel<<<(unsigned)(need < cap ? need : cap), IO_THREADS, 0, s>>>(c);
    return cudaGetLastError();
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
