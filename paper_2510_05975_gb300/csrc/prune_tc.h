// prune_tc.h -- Alg. 2 on whole-list pair tiles (k_prune_tc.cu): tcgen05 Gram tiles for 8-bit
// rows (K4 and the K6 first pass) and FP16 storage (K4), CUDA-core Gram blocks for other float
// rows (K4 and the K6 re-prune of listed sets).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cng_internal.h"
#include "prune_rule.cuh"

namespace cng {

// K4 on the Gram tile: fwd / fdeg as launch_prune_fwd writes them.
cudaError_t launch_prune_gram_u8(const uint8_t* U, int dw, const void* xs, int dtype, int64_t n,
                                 int d, int dpad, const int32_t* cand, const float* cdist, int L,
                                 const RuleArgs& ra, int32_t* fwd, int32_t* fdeg, Counters* ctr,
                                 cudaStream_t s);

// K4 on the Gram tile for FP16 rows (dpad 64 or 128, fixed rule): |x|^2 into norms[n], then the
// pipelined prune with certified decision windows.
cudaError_t launch_prune_gram_f16(const void* xs, int64_t n, int d, int dpad, const int32_t* cand,
                                  const float* cdist, int L, const RuleArgs& ra, int32_t* fwd,
                                  int32_t* fdeg, float* norms, Counters* ctr, cudaStream_t s);

// K4 for float rows on CUDA cores (lists of up to 256, fixed rule): all pairs of a list in
// 32 x 32 Gram blocks with certified decision windows, Alg. 2 on the masks.
cudaError_t launch_prune_pairs(const void* xs, int dtype, int64_t n, int d, int dpad,
                               const int32_t* cand, const float* cdist, int L, const RuleArgs& ra,
                               int32_t* fwd, int32_t* fdeg, Counters* ctr, cudaStream_t s);

// K6 re-prune of the float merged sets listed in ms (count ctr->nre) by the all-pairs kernel.
cudaError_t launch_merge_pairs(const void* xs, int dtype, int64_t n, int d, int dpad,
                               const MergeScratch& ms, const RuleArgs& ra, int32_t* adj, int32_t* deg,
                               Counters* ctr, cudaStream_t s);

// K6 first pass on the Gram tile: merged sets of up to 128 entries; larger ones are appended to
// mid_list (count in ctr->nmid) for the 256-entry pass.  With the fixed rule and scratch given
// (ms.mlist non-null) the sets are listed first and re-pruned by the pipelined Gram kernel.
cudaError_t launch_merge_gram_u8(const uint8_t* U, int dw, const void* xs, int dtype, int64_t n,
                                 int d, int dpad, const int32_t* fwd, const int32_t* fdeg,
                                 const int64_t* off, const int32_t* inl, const RuleArgs& ra,
                                 int32_t* adj, int32_t* deg, Counters* ctr, int32_t* mid_list,
                                 const MergeScratch& ms, cudaStream_t s);

}  // namespace cng
