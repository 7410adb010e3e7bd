// screen_tc.h -- tensor-core candidate screen (tcgen05 + TMA), host interface.
#pragma once

#include <stdint.h>

#include <string>

#include <cuda_runtime.h>

namespace cng {

struct TcScreenArgs {
  const void* A;      // rows   [m][kpad] bf16 (fp16 when fp16 != 0), zero padded
  const void* B;      // columns [n][kpad]
  int64_t m, n;
  int kpad;           // multiple of 64
  int fp16;
  const float* nb;    // ||y_b||^2 per column (length >= n rounded up to 256, zero padded)
  int Lp;             // screened list length per row
  int self_excl;      // 1: row i is column i and is skipped
  int32_t* ids;       // [m][Lp] screened ids (unordered), -1 padded
  uint32_t* thr;      // [m] ordered key of the largest kept score (0xffffffff: all kept)
  uint32_t* status;
  uint64_t* rowbuf;     // scratch: screen_tc_rowbuf_words(m, n, Lp) words
  size_t rowbuf_words;
  // Locality order (optional): A and B hold the points at positions of an order, perm[pos]
  // the point id; ids and thr are then written for the point ids (row perm[pos], column
  // perm[col]).  wave_start = 1 starts each wave of row blocks at its own column tile.
  const int32_t* perm;
  int wave_start;
  int64_t row_off = 0;  // position of row 0 in the order (tuning trials on a row sample)
  int variant = -1;     // pipeline variant; -1: the autotuner's choice
};

// Pipeline shape a screen ran with: variant index, operand stages, row-buffer capacity,
// checkpoint lag (windows of 256 tiles).
struct TcShape {
  int variant, stages, cap, sync_d;
};
int screen_tc_variants();
// The autotuned variant for a's shape (timing the variants on first use; synchronises `s`).
cudaError_t launch_screen_tc_tune(const TcScreenArgs& a, cudaStream_t s, std::string* msg, int* variant);

bool tc_screen_supported(int d, bool fp16);
// Scratch words for m rows against n columns: row buffers plus checkpoint counters.
size_t screen_tc_rowbuf_words(int64_t m, int64_t n, int Lp);
// The screen (launch on `s`); with a.variant < 0 the autotuned variant for this shape, timed
// on first use (synchronises `s` then).  *shape, if given, receives the shape used.
cudaError_t launch_screen_tc(const TcScreenArgs& a, cudaStream_t s, std::string* msg,
                             TcShape* shape = nullptr);
// Test aid: writes every screened score s(x, y) to dump[m][n] instead of selecting.
// One warp runs the screen's bounded waits on a barrier and a flag that never complete; they
// must run out and leave ST_TIMEOUT in *status (never_set: a zeroed device word).
cudaError_t launch_wait_probe(uint32_t* status, const uint32_t* never_set, cudaStream_t s);
cudaError_t launch_screen_tc_dump(const TcScreenArgs& a, float* dump, cudaStream_t s,
                                  std::string* msg);

}  // namespace cng
