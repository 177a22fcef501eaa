// k1_stencil_f32.cu -- float32 variant of the fused stencil (paper Sec. 2.2.1,
// Steps 1-3): sigma-parametrised Gaussian -> Sobel -> L2 strength -> direction
// sector -> non-maximum suppression, then the thresholds relative to the
// image's largest strength (a second, elementwise kernel, since the maximum is
// a grid-wide dependency). One CTA per output tile, staged in shared memory.
#include "canny_internal.cuh"

namespace canny {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ============================================================== float32 variant
// Same tiling; every product and sum is rounded separately (no contraction), in
// the order of the reference definition: taps accumulated from the first,
// horizontal pass before vertical, Sobel columns summed top to bottom.
constexpr int FTX = 32, FTY = 16;
constexpr int F_THREADS = 256;

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ int sector_f(float gx, float gy)
{
    const float t = 0.41421356f;
    float ax = fabsf(gx), ay = fabsf(gy);
    if (ay < fmul(ax, t)) return 0;
    if (ax < fmul(ay, t)) return 1;
    if ((gx > 0.f && gy > 0.f) || (gx < 0.f && gy < 0.f)) return 2;
    return 3;
}

__global__ void __launch_bounds__(F_THREADS)
k1f_magnitude_kernel(const uint8_t *__restrict__ in, int in_pitch, float *__restrict__ mag,
                     int mag_pitch, int w, int h, FloatParams fp, int nms, float *d_max)
{
    extern __shared__ float fsm[];
    const int R = fp.ksize / 2;
    const int inX = FTX + 2 * R + 4, inY = FTY + 2 * R + 4;
    const int sX = FTX + 4, sY = FTY + 4;
    const int mX = FTX + 2, mY = FTY + 2;
    float *I_s = fsm;                    // [inY][inX]
    float *H_s = I_s + inY * inX;        // [inY][sX]
    float *S_s = H_s + inY * sX;         // [sY][sX]
    float *GX_s = S_s + sY * sX;         // [mY][mX]
    float *GY_s = GX_s + mY * mX;
    float *M_s = GY_s + mY * mX;
    __shared__ float red[F_THREADS / 32];

    const int x0 = blockIdx.x * FTX, y0 = blockIdx.y * FTY;
    const int ox = x0 - R - 2, oy = y0 - R - 2;   // image coords of I_s[0][0] (clamped on read)
    const int tid = threadIdx.x;

    for (int i = tid; i < inX * inY; i += F_THREADS) {
        int r = i / inX, c = i % inX;
        int X = clampi(ox + c, 0, w - 1), Y = clampi(oy + r, 0, h - 1);
        I_s[r * inX + c] = (float)in[(int64_t)Y * in_pitch + X];
    }
    __syncthreads();
    // horizontal pass at columns X = clamp(x0-2+c)
    for (int i = tid; i < inY * sX; i += F_THREADS) {
        int r = i / sX, c = i % sX;
        int X = clampi(x0 - 2 + c, 0, w - 1);
        float acc = fmul(fp.taps[0], I_s[r * inX + (clampi(X - R, 0, w - 1) - ox)]);
        for (int k = 1; k < fp.ksize; ++k)
            acc = fadd(acc, fmul(fp.taps[k], I_s[r * inX + (clampi(X - R + k, 0, w - 1) - ox)]));
        H_s[r * sX + c] = acc;
    }
    __syncthreads();
    // vertical pass: S_s[r][c] = S(clamp(x0-2+c), clamp(y0-2+r))
    for (int i = tid; i < sY * sX; i += F_THREADS) {
        int r = i / sX, c = i % sX;
        int Y = clampi(y0 - 2 + r, 0, h - 1);
        float acc = fmul(fp.taps[0], H_s[(clampi(Y - R, 0, h - 1) - oy) * sX + c]);
        for (int k = 1; k < fp.ksize; ++k)
            acc = fadd(acc, fmul(fp.taps[k], H_s[(clampi(Y - R + k, 0, h - 1) - oy) * sX + c]));
        S_s[r * sX + c] = acc;
    }
    __syncthreads();
    // Sobel and strength on tile + ring
    float local_max = 0.f;
    for (int i = tid; i < mY * mX; i += F_THREADS) {
        int r = i / mX, c = i % mX;
        int X = x0 - 1 + c, Y = y0 - 1 + r;
        float gx = 0.f, gy = 0.f, m = 0.f;
        if (X >= 0 && X < w && Y >= 0 && Y < h) {
            int sr = r + 1, sc = c + 1;
#define SS(rr, cc) S_s[(rr) * sX + (cc)]
            float right = fadd(SS(sr - 1, sc + 1), fmul(2.f, SS(sr, sc + 1)));
            right = fadd(right, SS(sr + 1, sc + 1));
            float left = fadd(SS(sr - 1, sc - 1), fmul(2.f, SS(sr, sc - 1)));
            left = fadd(left, SS(sr + 1, sc - 1));
            float down = fadd(SS(sr + 1, sc - 1), fmul(2.f, SS(sr + 1, sc)));
            down = fadd(down, SS(sr + 1, sc + 1));
            float up = fadd(SS(sr - 1, sc - 1), fmul(2.f, SS(sr - 1, sc)));
            up = fadd(up, SS(sr - 1, sc + 1));
#undef SS
            gx = fadd(right, -left);
            gy = fadd(down, -up);
            m = __fsqrt_rn(fadd(fmul(gx, gx), fmul(gy, gy)));
            bool inner = r >= 1 && r <= FTY && c >= 1 && c <= FTX;
            if (inner) local_max = fmaxf(local_max, m);
        }
        GX_s[i] = gx;
        GY_s[i] = gy;
        M_s[i] = m;
    }
    // block max -> global max (non-negative floats order like their bit patterns)
    for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((tid & 31) == 0) red[tid >> 5] = local_max;
    __syncthreads();
    if (tid == 0) {
        float mx = 0.f;
        for (int k = 0; k < F_THREADS / 32; ++k) mx = fmaxf(mx, red[k]);
        if (d_max) atomicMax((unsigned int *)d_max, __float_as_uint(mx));
    }
    // output: strength, or strength after suppression (0 where suppressed)
    for (int i = tid; i < FTY * FTX; i += F_THREADS) {
        int r = i / FTX, c = i % FTX;
        int X = x0 + c, Y = y0 + r;
        if (X >= w || Y >= h) continue;
        int mr = r + 1, mc = c + 1;
        int k = mr * mX + mc;
        float m = M_s[k];
        if (nms) {
            int s = sector_f(GX_s[k], GY_s[k]);
            float mn, mp;
            if (s == 0) { mn = M_s[k - 1]; mp = M_s[k + 1]; }
            else if (s == 1) { mn = M_s[k - mX]; mp = M_s[k + mX]; }
            else if (s == 2) { mn = M_s[k - mX - 1]; mp = M_s[k + mX + 1]; }
            else { mn = M_s[k + mX - 1]; mp = M_s[k - mX + 1]; }
            bool keep = (m > mn) && (m >= mp);
            if (!keep) m = 0.f;
        }
        mag[(int64_t)Y * mag_pitch + X] = m;
    }
}

__global__ void k1f_classify_kernel(const float *__restrict__ mag, int mag_pitch,
                                    uint8_t *__restrict__ cls, int cls_pitch, int w, int h,
                                    const float *__restrict__ d_max, float lo_frac, float hi_frac)
{
    const float mmax = *d_max;
    const float lo_t = fmul(lo_frac, mmax), hi_t = fmul(hi_frac, mmax);
    int64_t n = (int64_t)w * h;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int y = (int)(i / w), x = (int)(i % w);
        float m = mag[(int64_t)y * mag_pitch + x];
        cls[(int64_t)y * cls_pitch + x] = m > hi_t ? 2 : (m > lo_t ? 1 : 0);
    }
}

}  // namespace

static size_t k1f_smem_bytes(int ksize)
{
    int R = ksize / 2;
    int inX = FTX + 2 * R + 4, inY = FTY + 2 * R + 4;
    int sX = FTX + 4, sY = FTY + 4, mX = FTX + 2, mY = FTY + 2;
    return sizeof(float) * ((size_t)inY * inX + (size_t)inY * sX + (size_t)sY * sX + 3 * (size_t)mY * mX);
}

cudaError_t launch_k1f_magnitude(const uint8_t *in, int in_pitch, float *mag, int mag_pitch,
                                 int w, int h, const FloatParams &fp, bool nms, float *d_max,
                                 cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    size_t smem = k1f_smem_bytes(fp.ksize);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k1f_magnitude_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)k1f_smem_bytes(MAX_KSIZE));
        attr_set = true;
    }
    dim3 grid((w + FTX - 1) / FTX, (h + FTY - 1) / FTY);
    k1f_magnitude_kernel<<<grid, F_THREADS, smem, s>>>(in, in_pitch, mag, mag_pitch, w, h, fp,
                                                       nms ? 1 : 0, d_max);
    return cudaGetLastError();
}

cudaError_t launch_k1f_classify(const float *mag_nms, int mag_pitch, uint8_t *cls, int cls_pitch,
                                int w, int h, const float *d_max, float lo_frac, float hi_frac,
                                cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    int64_t n = (int64_t)w * h;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k1f_classify_kernel<<<blocks, 256, 0, s>>>(mag_nms, mag_pitch, cls, cls_pitch, w, h, d_max,
                                               lo_frac, hi_frac);
    return cudaGetLastError();
}

}  // namespace canny
