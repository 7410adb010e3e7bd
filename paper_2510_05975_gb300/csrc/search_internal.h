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
  int* counter;         // SEARCH_COUNTER_INTS work-queue words, zeroed before launch
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
  int min_stable;           // the model is consulted only when hops - tlc >= min_stable
  // per-query exactness when the data is exact (exact != 0): qflag[q] == 0 marks an integer
  // query inside the data's range; other queries resolve near-ties in FP64 (unused with qids)
  const uint8_t* qflag;
  // 8-bit rows (integer data spanning <= 255, shifted by the data minimum): exact queries use
  // exact integer squared distances from 4 u8w-byte rows instead of FP32 rows; null: FP32
  const uint8_t* U;         // [n][4 u8w]
  const uint8_t* QU;        // queries in the same form [nq][4 u8w] (unused with qids)
  int u8w;                  // 8, 16, 24 or 32
  // two-kernel launch (SearchPlan::fast_qs > 0): the register-queue kernel serves every exact
  // query and appends the others to defer[] (>= nq entries, counter[1] counts them); the general
  // kernel then serves the list qlist[0 .. *nq_dev) with counter[2] as its queue head
  int32_t* defer;
  const int32_t* qlist;
  const int* nq_dev;
  size_t warp_smem_fast;    // bytes of shared memory per warp of the register-queue kernel
};

constexpr int SEARCH_COUNTER_INTS = 4;

// Launch shape of one batched search.  fast_qs > 0: the register-queue kernel (queue of up to
// 32 * fast_qs entries in registers; data with 8-bit rows) runs first on `grid` blocks, then the
// general kernel on `grid_defer` blocks for the deferred queries; fast_qs == 0: the general
// kernel alone on `grid` blocks.
struct SearchPlan {
  int wpb = 0;
  int grid = 0;
  int fast_qs = 0;
  int grid_defer = 0;
  int wpb_defer = 0;
};

// Packed stop model for inference: W1 bf16 [64][24] (row o = W1[o][0..15], then 8 pad), W2
// bf16 [64][72] (row o = W2[o][0..63], then 8 pad), then floats b1[64] b2[64] w3[64] b3[1]
// pad[3] mu[16] sigma[16].
constexpr int STOP_BLOCK_BYTES = 64 * 24 * 2 + 64 * 72 * 2 + (64 * 3 + 4 + 32) * 4;

size_t search_warp_smem(int dpad, int L, int hash_slots);
// Plans a search of `a` (its L, U/u8w, exact, model set) with wpb warps per block and a visited
// filter of hash_slots entries: fills a.hash_slots, a.warp_smem, a.warp_smem_fast and *p and sets
// the kernels' shared-memory attributes, so call it outside any stream capture.  Returns false
// if the shape does not fit.
bool search_plan(SearchArgs& a, int wpb, int hash_slots, SearchPlan* p);
cudaError_t launch_search(const SearchArgs& a, const SearchPlan& p, cudaStream_t s);
// Per-query exactness flags (0: integer query inside [vmin, vmax]) and, with out != null, the
// queries as 8-bit rows out[q][c] = x[q][c] - vmin.
cudaError_t launch_query_check(const float* Q, int64_t nq, int d, float vmin, float vmax, int u8w,
                               uint8_t* out, uint8_t* flag, cudaStream_t s);
// Blocks per SM of the general search kernel for (dtype, u8w: 0 = FP32 path), and of the
// register-queue kernel for (u8w, qs, learn: the variant with stop features); both also set
// the kernel's shared-memory attribute.
int search_blocks_per_sm(int dtype, int u8w, int warps_per_block, size_t smem);
int search_fast_blocks_per_sm(int u8w, int qs, bool learn, int warps_per_block, size_t smem);
size_t search_fast_warp_smem(int u8w, int hash_slots);
cudaError_t launch_search_general(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t s);
cudaError_t launch_search_fast(const SearchArgs& a, int qs, int warps_per_block, int grid, cudaStream_t s);

}  // namespace cng
