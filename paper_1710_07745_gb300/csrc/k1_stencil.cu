// k1_stencil.cu -- fused Steps 1-3 + double threshold (paper Sec. 2.2.1):
// Gaussian -> Sobel -> strength -> direction sector -> non-maximum suppression
// -> class map (0 none, 1 weak, 2 strong). One CTA per output tile; the tile and
// its halo are staged in shared memory and nothing but the input and the class
// map touches HBM.
#include "canny_internal.cuh"

namespace canny {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// ============================================================== integer path
constexpr int TX = 64, TY = 16;            // output tile
constexpr int IN_X = TX + 8, IN_Y = TY + 8;  // input tile: halo 2 (Gauss) + 1 (Sobel) + 1 (NMS)
constexpr int SX = TX + 4, SY = TY + 4;      // smoothed tile
constexpr int MX = TX + 2, MY = TY + 2;      // strength tile
constexpr int K1_THREADS = 256;

// Q15 tan(22.5 deg) for the sector test: round((sqrt(2) - 1) * 2^15).
constexpr int TAN_Q15 = 13573;

__global__ void __launch_bounds__(K1_THREADS)
k1_classify_u8_kernel(const uint8_t *__restrict__ in, int in_pitch, uint8_t *__restrict__ cls,
                      int cls_pitch, int w, int h, IntThresholds t)
{
    __shared__ uint8_t I_s[IN_Y][IN_X];
    __shared__ int H_s[IN_Y][SX];
    __shared__ uint8_t S_s[SY][SX];
    __shared__ int M_s[MY][MX];

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;

    // input with replicate border: I_s[r][c] = I(clamp(x0-4+c), clamp(y0-4+r))
    for (int i = tid; i < IN_X * IN_Y; i += K1_THREADS) {
        int r = i / IN_X, c = i % IN_X;
        int X = clampi(x0 - 4 + c, 0, w - 1), Y = clampi(y0 - 4 + r, 0, h - 1);
        I_s[r][c] = in[(int64_t)Y * in_pitch + X];
    }
    __syncthreads();

    // Step 1, horizontal binomial pass at columns X = clamp(x0-2+c)
    for (int i = tid; i < IN_Y * SX; i += K1_THREADS) {
        int r = i / SX, c = i % SX;
        int X = clampi(x0 - 2 + c, 0, w - 1);
        int base = X - (x0 - 4);
        int a0 = I_s[r][clampi(X - 2, 0, w - 1) - (x0 - 4)];
        int a1 = I_s[r][clampi(X - 1, 0, w - 1) - (x0 - 4)];
        int a2 = I_s[r][base];
        int a3 = I_s[r][clampi(X + 1, 0, w - 1) - (x0 - 4)];
        int a4 = I_s[r][clampi(X + 2, 0, w - 1) - (x0 - 4)];
        H_s[r][c] = a0 + 4 * a1 + 6 * a2 + 4 * a3 + a4;
    }
    __syncthreads();

    // Step 1, vertical pass and rounding: S_s[r][c] = S(clamp(x0-2+c), clamp(y0-2+r))
    for (int i = tid; i < SY * SX; i += K1_THREADS) {
        int r = i / SX, c = i % SX;
        int Y = clampi(y0 - 2 + r, 0, h - 1);
        int acc = 0;
        const int wts[5] = {1, 4, 6, 4, 1};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            int Yk = clampi(Y - 2 + k, 0, h - 1);
            acc += wts[k] * H_s[Yk - (y0 - 4)][c];
        }
        S_s[r][c] = (uint8_t)((acc + 128) >> 8);
    }
    __syncthreads();

    // Step 2, Sobel strength on the tile plus a 1-pixel ring (0 outside the image)
    for (int i = tid; i < MY * MX; i += K1_THREADS) {
        int r = i / MX, c = i % MX;
        int X = x0 - 1 + c, Y = y0 - 1 + r;
        int m2 = 0;
        if (X >= 0 && X < w && Y >= 0 && Y < h) {
            int sr = r + 1, sc = c + 1;   // S_s index of (X, Y)
            int gx = (S_s[sr - 1][sc + 1] + 2 * S_s[sr][sc + 1] + S_s[sr + 1][sc + 1]) -
                     (S_s[sr - 1][sc - 1] + 2 * S_s[sr][sc - 1] + S_s[sr + 1][sc - 1]);
            int gy = (S_s[sr + 1][sc - 1] + 2 * S_s[sr + 1][sc] + S_s[sr + 1][sc + 1]) -
                     (S_s[sr - 1][sc - 1] + 2 * S_s[sr - 1][sc] + S_s[sr - 1][sc + 1]);
            m2 = gx * gx + gy * gy;
        }
        M_s[r][c] = m2;
    }
    __syncthreads();

    // Step 3 + thresholds on the output tile
    for (int i = tid; i < TY * TX; i += K1_THREADS) {
        int r = i / TX, c = i % TX;
        int X = x0 + c, Y = y0 + r;
        if (X >= w || Y >= h) continue;
        int sr = r + 2, sc = c + 2;
        int gx = (S_s[sr - 1][sc + 1] + 2 * S_s[sr][sc + 1] + S_s[sr + 1][sc + 1]) -
                 (S_s[sr - 1][sc - 1] + 2 * S_s[sr][sc - 1] + S_s[sr + 1][sc - 1]);
        int gy = (S_s[sr + 1][sc - 1] + 2 * S_s[sr + 1][sc] + S_s[sr + 1][sc + 1]) -
                 (S_s[sr - 1][sc - 1] + 2 * S_s[sr - 1][sc] + S_s[sr - 1][sc + 1]);
        int ax = abs(gx), ay = abs(gy);
        int mr = r + 1, mc = c + 1;
        int m = M_s[mr][mc];
        int mn, mp;
        if (ay * 32768 < ax * TAN_Q15) {            // H: left / right
            mn = M_s[mr][mc - 1]; mp = M_s[mr][mc + 1];
        } else if (ax * 32768 < ay * TAN_Q15) {     // V: up / down
            mn = M_s[mr - 1][mc]; mp = M_s[mr + 1][mc];
        } else if ((gx > 0 && gy > 0) || (gx < 0 && gy < 0)) {  // D: up-left / down-right
            mn = M_s[mr - 1][mc - 1]; mp = M_s[mr + 1][mc + 1];
        } else {                                     // A: down-left / up-right
            mn = M_s[mr + 1][mc - 1]; mp = M_s[mr - 1][mc + 1];
        }
        bool keep = (m > mn) && (m >= mp);
        uint8_t v = 0;
        if (keep && m > t.hi2) v = 2;
        else if (keep && m > t.lo2) v = 1;
        cls[(int64_t)Y * cls_pitch + X] = v;
    }
}

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

cudaError_t launch_k1_classify_u8(const uint8_t *in, int in_pitch, uint8_t *cls, int cls_pitch,
                                  int w, int h, IntThresholds t, cudaStream_t s)
{
    if (w <= 0 || h <= 0) return cudaSuccess;
    dim3 grid((w + TX - 1) / TX, (h + TY - 1) / TY);
    k1_classify_u8_kernel<<<grid, K1_THREADS, 0, s>>>(in, in_pitch, cls, cls_pitch, w, h, t);
    return cudaGetLastError();
}

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
