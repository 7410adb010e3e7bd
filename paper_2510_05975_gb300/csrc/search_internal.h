// search_internal.h -- argument block of the batched search kernel (host and device).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

namespace cng {

struct SearchArgs {
  const void* X;        // stored points [n][dpad] (float or half)
  int dtype;
  int64_t n;
  int d, dpad;
  const int32_t* adj;   // [n][R]
  const int32_t* deg;   // [n]
  int R;
  int32_t entry;
  const float* Q;       // queries [nq][d]
  int64_t nq;
  int k, L;
  int hash_slots;       // power of two
  size_t warp_smem;     // bytes of shared memory per warp
  float band;
  int exact;
  int max_hops;
  int* counter;         // work queue head (zeroed before launch)
  int32_t* ids;
  float* dists;
  int32_t* ndc;
  int32_t* hops;
  int32_t* flags;
  unsigned long long* tot;  // [4]: ndc, hops, fp64 decisions, learned stops
  uint32_t* status;         // device status word (ST_* bits)
};

size_t search_warp_smem(int dpad, int L, int hash_slots);
cudaError_t launch_search(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t s);
int search_blocks_per_sm(int dtype, int warps_per_block, size_t smem);

}  // namespace cng
