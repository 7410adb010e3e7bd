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
  const int32_t* qids;  // or: query i is stored point qids[i] (Q unused)
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
  // learned early stop
  float* trace_feats;       // [nq][max_trace][16] per-hop features, or null
  int max_trace;
  int32_t* tlc;             // [nq] last hop at which the top-k list changed, or null
  const void* model;        // packed stop model (STOP_BLOCK_BYTES), or null
  float zthr;               // stop when the logit >= zthr
  int check_every;
  // per-query exactness when the data is exact (exact != 0): qflag[q] == 0 marks an integer
  // query inside the data's range; other queries resolve near-ties in FP64 (unused with qids)
  const uint8_t* qflag;
  // 8-bit rows (integer data spanning <= 255, shifted by the data minimum): exact queries use
  // exact integer squared distances from 4 u8w-byte rows instead of FP32 rows; null: FP32
  const uint8_t* U;         // [n][4 u8w]
  const uint8_t* QU;        // queries in the same form [nq][4 u8w] (unused with qids)
  int u8w;                  // 8, 16, 24 or 32
};

// Packed stop model for inference: W1T bf16 [16][64], W2T bf16 [64][64], then floats
// b1[64] b2[64] w3[64] b3[1] pad[3] mu[16] sigma[16].
constexpr int STOP_BLOCK_BYTES = 16 * 64 * 2 + 64 * 64 * 2 + (64 * 3 + 4 + 32) * 4;

size_t search_warp_smem(int dpad, int L, int hash_slots);
cudaError_t launch_search(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t s);
// Per-query exactness flags (0: integer query inside [vmin, vmax]) and, with out != null, the
// queries as 8-bit rows out[q][c] = x[q][c] - vmin.
cudaError_t launch_query_check(const float* Q, int64_t nq, int d, float vmin, float vmax, int u8w,
                               uint8_t* out, uint8_t* flag, cudaStream_t s);
// Blocks per SM of the search variant for (dtype, u8w: 0 = FP32 path); also sets its
// shared-memory attribute, so call it before launching (outside any stream capture).
int search_blocks_per_sm(int dtype, int u8w, int warps_per_block, size_t smem);

}  // namespace cng
