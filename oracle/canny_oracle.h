/*
 * canny_oracle.h -- plain, single-threaded CPU Canny edge detector.
 *
 * TEST INFRASTRUCTURE. This is the checker that the CUDA library is compared
 * against, not part of the product. Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference legs may load or call it. It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * It computes every stage of the four-step pipeline of "High Performance Canny
 * Edge Detector using Parallel Patterns" (Mogale), Sec. 2.2.1, Steps 1-4, over
 * the whole image into full-size arrays, in the order the paper lists them:
 * Gaussian noise filter, Sobel gradient strength and direction, non-maximum
 * suppression, hysteresis. The paper leaves the constants open; the readings
 * used here (5x5 binomial, replicate borders, 4-sector fixed-point direction,
 * strict thresholds, 8-connectivity, the fp32 variant's operation order) are
 * stated at each function.
 *
 * Every function is pinned by tests/test_oracle_*.py against closed forms,
 * library routines (numpy/scipy), brute force and invariants; none is
 * "parity unpinned".
 */
#ifndef CANNY_ORACLE_H
#define CANNY_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* direction sectors of the non-maximum suppression (Step 3) */
enum { ORACLE_SECTOR_H = 0, ORACLE_SECTOR_V = 1, ORACLE_SECTOR_D = 2, ORACLE_SECTOR_A = 3 };
/* class map values between thresholding and hysteresis (Step 4) */
enum { ORACLE_NONE = 0, ORACLE_WEAK = 1, ORACLE_STRONG = 2 };

/* ---------------- integer path ---------------- */
void oracle_gauss5_u8(const uint8_t *img, int w, int h, int pitch, uint8_t *S);
void oracle_sobel_u8(const uint8_t *S, int w, int h, int16_t *gx, int16_t *gy);
void oracle_mag2_i32(const int16_t *gx, const int16_t *gy, int64_t n, int32_t *m2);
int  oracle_sector_tan_q15(void);
int  oracle_sector_i(int gx, int gy);
void oracle_sector_map_i(const int32_t *gx, const int32_t *gy, int64_t n, uint8_t *sec);
void oracle_nms_classify_u8(const int16_t *gx, const int16_t *gy, const int32_t *m2,
                            int w, int h, int64_t lo2, int64_t hi2, uint8_t *cls);
void oracle_hysteresis(const uint8_t *cls, int w, int h, uint8_t *out, int out_pitch);
void oracle_classify_u8(const uint8_t *img, int w, int h, int pitch, int low, int high,
                        uint8_t *cls);
void oracle_canny_u8(const uint8_t *img, int w, int h, int in_pitch, int low, int high,
                     uint8_t *out, int out_pitch);

/* ---------------- float32 variant ---------------- */
void  oracle_gauss_taps_f32(float sigma, int ksize, float *taps);
void  oracle_gauss_f32(const uint8_t *img, int w, int h, int pitch, float sigma, int ksize,
                       float *S);
void  oracle_sobel_f32(const float *S, int w, int h, float *gx, float *gy);
void  oracle_magnitude_f32(const float *gx, const float *gy, int64_t n, float *M);
float oracle_max_f32(const float *M, int64_t n);
int   oracle_sector_f(float gx, float gy);
void  oracle_nms_classify_f32(const float *gx, const float *gy, const float *M, int w, int h,
                              float lo_t, float hi_t, uint8_t *cls);
void  oracle_canny_f32(const uint8_t *img, int w, int h, int in_pitch, float sigma, int ksize,
                       float lo_frac, float hi_frac, uint8_t *out, int out_pitch,
                       float *M_out, uint8_t *cls_out);

#ifdef __cplusplus
}
#endif
#endif
