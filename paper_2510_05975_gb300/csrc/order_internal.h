// order_internal.h -- locality order of the point set (k_order.cu), host interface.
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

namespace cng {

// Levels of median splits for n points (segments end with at most 256 points).
int order_levels(int64_t n);
// Device scratch launch_order needs for n points.
size_t order_scratch_bytes(int64_t n);
// perm[p] = id of the point at position p of the k-d order of xs [n][dpad] (f32 or f16).
cudaError_t launch_order(const void* xs, int dtype, int64_t n, int d, int dpad, int32_t* perm,
                         void* scratch, cudaStream_t s);
// xo[p] = xi[perm[p]] for rows of kpad 16-bit values, nbo[p] = nbi[perm[p]].
cudaError_t launch_order_gather(const void* xi, const float* nbi, const int32_t* perm, int64_t n,
                                int kpad, void* xo, float* nbo, cudaStream_t s);

}  // namespace cng
