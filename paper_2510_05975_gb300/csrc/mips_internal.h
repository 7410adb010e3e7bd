// mips_internal.h -- the inner-product augmentation kernels (host declarations).
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

namespace cng {

// out [n][d + 1] f32 = [x, sqrt(M^2 - |x|^2)] with |x|^2 summed in FP64 in coordinate order and
// M^2 = max |x|^2; nrm2 [n] and max_bits (M^2 as its bit pattern) are scratch.  X: f32 or f16
// [n][d] (dtype CNG_F32 / CNG_F16), device memory.
cudaError_t launch_mips_augment(const void* X, int dtype, int64_t n, int d, double* nrm2,
                                unsigned long long* max_bits, float* out, cudaStream_t s);
// out [nq][d + 1] = [q, 0].
cudaError_t launch_append_zero(const float* Q, int64_t nq, int d, float* out, cudaStream_t s);

}  // namespace cng
