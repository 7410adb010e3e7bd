/*
 * cng_debug.h -- test aids exported by libcng.so (not part of the alpha-CNG method).
 */
#ifndef CNG_DEBUG_H_
#define CNG_DEBUG_H_

#include <stdint.h>

#include "cng.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * cngx_tc_scores -- run the tensor-core screen's MMA and epilogue arithmetic on m rows and n
 * columns (f32 device arrays, row-major, d columns, d <= 192) and write every screened score
 * s(x, y) = ||y_b||^2 - 2 <x_b, y_b> (x_b, y_b: bf16-rounded rows) to scores_dev [m][n] (f32,
 * device).  Lets tests compare the tcgen05 pipeline with a plain reference of the same
 * arithmetic.  Synchronises `stream`.
 */
cng_status cngx_tc_scores(const float *rows_dev, int64_t m, const float *cols_dev, int64_t n,
                          int32_t d, float *scores_dev, void *stream);

/*
 * cngx_tc_scores_f16 -- as cngx_tc_scores with the operands the build uses for f32 data:
 * x_b = fp16(scale * x), y_b = fp16(scale * y) (scale a power of two, else CNG_E_INVAL), so the
 * scores are in units of scale^2.
 */
cng_status cngx_tc_scores_f16(const float *rows_dev, int64_t m, const float *cols_dev, int64_t n,
                              int32_t d, float scale, float *scores_dev, void *stream);

/* Number of CUDA kernel launches this library has issued since it was loaded (each launch
 * site counts once per launch). */
long long cngx_launches(void);

/*
 * cngx_wait_probe -- failure-path check of the tensor-core screen's bounded waits: one warp
 * waits on an mbarrier nothing arrives on and polls a device word nothing sets, each with the
 * screen's own bounded wait; both must run out.  *status_out receives the device status word:
 * bit 0 (timeout) set and bit 3 clear when the waits expired as designed.  Synchronises the
 * device; the context stays usable.
 */
cng_status cngx_wait_probe(uint32_t *status_out);

#ifdef __cplusplus
}
#endif
#endif /* CNG_DEBUG_H_ */
