/*
 * synth.c -- seeded synthetic grayscale images for the Canny pipeline.
 *
 * Input generator only: it holds none of the edge detector's arithmetic and
 * is the one piece of code that both the CPU oracle and the CUDA library are
 * fed from (the same bytes go to both). The paper measures on photographs it
 * does not publish (Sec. 2.2, Fig. 7); these images stand in for them: a
 * smooth linear gradient, filled rectangles and disks of uniform random
 * intensity, additive noise, clamped to [0, 255].
 *
 * Arithmetic is integer-only, so a seed gives the same bytes on every host:
 *   - random numbers: a counter-based generator, value k of stream key is
 *     mix64(key + (k + 1) * 0x9E3779B97F4A7C15), where mix64 is the SplitMix64
 *     output function (Steele, Lea, Flood, "Fast splittable pseudorandom number
 *     generators", OOPSLA 2014);
 *   - background: v = round(255 * (p - pmin) / (pmax - pmin)) with
 *     p = a*x + b*y and (a, b) a random integer direction in [-256, 256]^2;
 *   - rectangles: centre uniform over the image, sides uniform in
 *     [max(2, S/64), max(3, S/4)] (S = that image dimension), painted in order;
 *   - disks, painted after the rectangles: centre uniform, radius uniform in
 *     [max(1, m/64), max(2, m/8)], m = min(w, h), pixels with
 *     dx^2 + dy^2 <= r^2;
 *   - noise: sigma * N, where N is the Irwin-Hall sum of twelve uniform 16-bit
 *     draws minus its mean (variance 1 in units of 2^16), rounded to nearest
 *     and clamped.
 * Rows are split into bands across threads; every value depends only on
 * (seed, position), so the bytes do not depend on the thread count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t ctr)
{
    return mix64(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

/* uniform integer in [lo, hi] (inclusive) from one 64-bit draw (multiply-high) */
static inline int64_t uni(uint64_t key, uint64_t *ctr, int64_t lo, int64_t hi)
{
    uint64_t span = (uint64_t)(hi - lo) + 1;
    unsigned __int128 m = (unsigned __int128)draw(key, (*ctr)++) * span;
    return lo + (int64_t)(uint64_t)(m >> 64);
}

static inline int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

static inline int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }
static inline int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }

typedef struct { int x0, x1, y0, y1, v; } rect_t;          /* half-open */
typedef struct { int cx, cy, r, v; } disk_t;

typedef struct {
    uint8_t *out;
    int w, h, pitch, y_begin, y_end;
    int64_t a, b, pmin, pmax;
    const rect_t *rects;
    int n_rect;
    const disk_t *disks;
    int n_disk;
    int noise_sigma;
    uint64_t noise_key;
} band_t;

static int64_t isqrt64(int64_t v)
{
    if (v <= 0) return 0;
    int64_t r = 0, bit = (int64_t)1 << 62;
    while (bit > v) bit >>= 2;
    while (bit) {
        if (v >= r + bit) { v -= r + bit; r = (r >> 1) + bit; }
        else r >>= 1;
        bit >>= 2;
    }
    return r;
}

static void *paint_band(void *arg)
{
    band_t *B = (band_t *)arg;
    const int64_t den = B->pmax - B->pmin;
    for (int y = B->y_begin; y < B->y_end; ++y) {
        uint8_t *row = B->out + (int64_t)y * B->pitch;
        for (int x = 0; x < B->w; ++x) {
            int64_t v = 128;
            if (den > 0) v = (255 * (B->a * x + B->b * y - B->pmin) * 2 + den) / (2 * den);
            row[x] = (uint8_t)v;
        }
    }
    for (int k = 0; k < B->n_rect; ++k) {
        const rect_t *R = &B->rects[k];
        int y0 = (int)imax(R->y0, B->y_begin), y1 = (int)imin(R->y1, B->y_end);
        for (int y = y0; y < y1; ++y)
            memset(B->out + (int64_t)y * B->pitch + R->x0, R->v, (size_t)(R->x1 - R->x0));
    }
    for (int k = 0; k < B->n_disk; ++k) {
        const disk_t *D = &B->disks[k];
        int y0 = (int)imax((int64_t)D->cy - D->r, B->y_begin);
        int y1 = (int)imin((int64_t)D->cy + D->r + 1, B->y_end);
        for (int y = y0; y < y1; ++y) {
            int64_t dy = y - D->cy;
            int64_t dx = isqrt64((int64_t)D->r * D->r - dy * dy);
            int64_t x0 = imax(D->cx - dx, 0), x1 = imin(D->cx + dx + 1, B->w);
            if (x1 > x0) memset(B->out + (int64_t)y * B->pitch + x0, D->v, (size_t)(x1 - x0));
        }
    }
    if (B->noise_sigma > 0) {
        for (int y = B->y_begin; y < B->y_end; ++y) {
            uint8_t *row = B->out + (int64_t)y * B->pitch;
            for (int x = 0; x < B->w; ++x) {
                uint64_t idx = (uint64_t)y * (uint64_t)B->w + (uint64_t)x;
                int64_t s = 0;
                for (int k = 0; k < 3; ++k) {
                    uint64_t r = draw(B->noise_key, 3 * idx + (uint64_t)k);
                    s += (int64_t)(r & 0xFFFF) + (int64_t)((r >> 16) & 0xFFFF) +
                         (int64_t)((r >> 32) & 0xFFFF) + (int64_t)(r >> 48);
                }
                s -= 6 * 65535;                       /* 12 draws, mean 65535/2 each */
                int64_t v = floordiv(((int64_t)row[x] << 16) + s * B->noise_sigma + 32768, 65536);
                row[x] = (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
            }
        }
    }
    return NULL;
}

/*
 * Fill out (h rows of w bytes, row stride pitch) with the image of the given
 * seed. Returns 0, or -1 on bad arguments / allocation failure.
 */
int synth_image(uint64_t seed, int w, int h, int pitch, int n_rect, int n_disk,
                int noise_sigma, int n_threads, uint8_t *out)
{
    if (w < 0 || h < 0 || pitch < w || n_rect < 0 || n_disk < 0 || noise_sigma < 0 || !out)
        return -1;
    if (w == 0 || h == 0) return 0;
    const uint64_t key_bg = mix64(seed ^ 0x6267000000000001ULL);
    const uint64_t key_obj = mix64(seed ^ 0x6f626a0000000002ULL);
    const uint64_t key_noise = mix64(seed ^ 0x6e6f697365000003ULL);

    uint64_t c = 0;
    int64_t a, b;
    do {
        a = uni(key_bg, &c, -256, 256);
        b = uni(key_bg, &c, -256, 256);
    } while (a == 0 && b == 0);
    int64_t corners[4] = {0, a * (w - 1), b * (h - 1), a * (w - 1) + b * (h - 1)};
    int64_t pmin = corners[0], pmax = corners[0];
    for (int k = 1; k < 4; ++k) {
        pmin = imin(pmin, corners[k]);
        pmax = imax(pmax, corners[k]);
    }

    rect_t *rects = (rect_t *)malloc(sizeof(rect_t) * (size_t)(n_rect ? n_rect : 1));
    disk_t *disks = (disk_t *)malloc(sizeof(disk_t) * (size_t)(n_disk ? n_disk : 1));
    if (!rects || !disks) { free(rects); free(disks); return -1; }
    c = 0;
    for (int k = 0; k < n_rect; ++k) {
        int64_t cx = uni(key_obj, &c, 0, w - 1), cy = uni(key_obj, &c, 0, h - 1);
        int64_t sw = uni(key_obj, &c, imax(2, w / 64), imax(3, w / 4));
        int64_t sh = uni(key_obj, &c, imax(2, h / 64), imax(3, h / 4));
        int v = (int)uni(key_obj, &c, 0, 255);
        rect_t R;
        R.x0 = (int)imax(cx - sw / 2, 0);
        R.x1 = (int)imin(cx - sw / 2 + sw, w);
        R.y0 = (int)imax(cy - sh / 2, 0);
        R.y1 = (int)imin(cy - sh / 2 + sh, h);
        R.v = v;
        if (R.x1 < R.x0) R.x1 = R.x0;
        if (R.y1 < R.y0) R.y1 = R.y0;
        rects[k] = R;
    }
    int64_t m = imin(w, h);
    for (int k = 0; k < n_disk; ++k) {
        disk_t D;
        D.cx = (int)uni(key_obj, &c, 0, w - 1);
        D.cy = (int)uni(key_obj, &c, 0, h - 1);
        D.r = (int)uni(key_obj, &c, imax(1, m / 64), imax(2, m / 8));
        D.v = (int)uni(key_obj, &c, 0, 255);
        disks[k] = D;
    }

    if (n_threads < 1) n_threads = 1;
    if (n_threads > h) n_threads = h;
    if (n_threads > 256) n_threads = 256;
    band_t bands[256];
    pthread_t tid[256];
    for (int t = 0; t < n_threads; ++t) {
        band_t *B = &bands[t];
        B->out = out; B->w = w; B->h = h; B->pitch = pitch;
        B->y_begin = (int)((int64_t)h * t / n_threads);
        B->y_end = (int)((int64_t)h * (t + 1) / n_threads);
        B->a = a; B->b = b; B->pmin = pmin; B->pmax = pmax;
        B->rects = rects; B->n_rect = n_rect; B->disks = disks; B->n_disk = n_disk;
        B->noise_sigma = noise_sigma; B->noise_key = key_noise;
    }
    int started = 0;
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&tid[t], NULL, paint_band, &bands[t]) != 0) break;
        started = t;
    }
    paint_band(&bands[0]);
    for (int t = started + 1; t < n_threads; ++t) paint_band(&bands[t]); /* threads not started */
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    free(rects);
    free(disks);
    return 0;
}

/*
 * n image sizes with width and height drawn independently and log-uniformly
 * in [lo, hi]: side = floor(lo * (hi/lo)^u + 1/2), u uniform in [0, 1) with 53
 * random bits. pow() is the host libm's; sizes are inputs, not checked values.
 */
#include <math.h>
void synth_log_uniform_sizes(uint64_t seed, int n, int lo, int hi, int *ws, int *hs)
{
    const uint64_t key = mix64(seed ^ 0x73697a6500000004ULL);
    double ratio = (double)hi / (double)lo;
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 2; ++k) {
            double u = (double)(draw(key, 2 * (uint64_t)i + (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
            int64_t s = (int64_t)floor((double)lo * pow(ratio, u) + 0.5);
            if (s < lo) s = lo;
            if (s > hi) s = hi;
            (k == 0 ? ws : hs)[i] = (int)s;
        }
    }
}

/* n exponential inter-arrival gaps (Poisson process) with mean 1/rate, in seconds. */
void synth_poisson_arrivals(uint64_t seed, int n, double rate, double *t_out)
{
    const uint64_t key = mix64(seed ^ 0x6172727600000005ULL);
    double t = 0.0;
    for (int i = 0; i < n; ++i) {
        double u = ((double)(draw(key, (uint64_t)i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        t += -log(u) / rate;
        t_out[i] = t;
    }
}
