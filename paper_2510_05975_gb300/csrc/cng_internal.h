// cng_internal.h -- host-side declarations shared by the libcng translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include <string>

#include "../../include/cng.h"
#include "status_bits.h"

namespace cng {

// Statistics written by the preparation kernel (device memory, one per build).
struct PrepStats {
  uint32_t nonint;        // != 0 if some coordinate is not an integer
  uint32_t vmin_key;      // ordered-key min / max over all coordinates
  uint32_t vmax_key;
  uint32_t nbmax_bits;    // max squared norm of the screening operand (float bits, >= 0)
  uint32_t rbmax_bits;    // max ||bf16(x) - x||
  uint32_t normmax_bits;  // max ||x||
  uint32_t unitdev_bits;  // max | ||x|| - 1 |
  uint32_t pad;
};

// Device counters accumulated by the build kernels.
struct Counters {
  unsigned long long order_ties;
  unsigned long long rule_ties;
  unsigned long long merge_repruned;
  unsigned long long merge_max_list;
  unsigned long long edges;
  int nfail;
  uint32_t status;
  uint32_t screen_err_bits;
  int nbig;        // nodes whose merged set exceeds the shared-memory capacity
  int max_indeg;
  int nmid;        // 8-bit merge: nodes deferred from the 128-entry to the 256-entry pass
  unsigned long long alpha_steps;  // adaptive pruning: sum over phase-2 points of the alpha step
  int nre;         // 8-bit merge: nodes listed for the pipelined Gram re-prune
};

// Scratch of the merge's re-prune by the Gram-tile / all-pairs kernels: merged lists in (D, id)
// order of up to `stride` entries per node ([n][stride] ids and FP32 distances; 128 for 8-bit
// rows, 256 for float rows), their lengths and the listed nodes.  All null: not used.
struct MergeScratch {
  int32_t* mlist;
  float* mdist;
  int32_t* mlen;
  int32_t* rlist;
  int stride;
};

// Alg. 4 grid of adaptive pruning: alpha_i = alpha0 + i * dalpha, i = 0 .. imax (imax < 0:
// the fixed alpha of Alg. 2 everywhere).
struct AlphaGrid {
  double alpha0, dalpha;
  int imax;
};

// How the screened score relates to the squared distance (for certification).
struct ScreenModel {
  int kind;          // 0: FP32 direct squared distance; 1: tensor-core shifted score
  int exact;         // 1: scores are exact integers
  float rel_err;     // kind 0: relative error bound of the screened squared distance
  const float* nb;   // kind 1: ||x_b||^2 per point (shift of the score)
  const float* rb;   // kind 1: ||x_b - x|| per point
  float rbmax;       // kind 1: max rb
  float acc_err;     // kind 1: absolute accumulation error bound per unit of (||x||+||y||)^2
  float normmax;     // kind 1: max ||x_b||
  float scale2;      // kind 1: the operands are x_b ~ s x; scores are in units of s^2 (a power of 4)
};

// Launchers (each returns cudaError_t of the launch).
// out[0] = bits of max |x|, out[1] != 0 if some coordinate is not an integer (out pre-zeroed).
cudaError_t launch_absmax(const void* pts, int dtype, int64_t n, int d, uint32_t* out,
                          cudaStream_t s);
// xb_* receive round(scale * x) (scale a power of two); nb, rb are in those units.
cudaError_t launch_prep(const void* pts, int dtype, int64_t n, int d, int dpad, void* xs,
                        __nv_bfloat16* xb_bf, __half* xb_h, int kpad, float* nb, float* rb,
                        float scale,
                        PrepStats* st, cudaStream_t s);
cudaError_t launch_entry(const void* xs, int dtype, int64_t n, int d, int dpad, double* part,
                         double* cen, unsigned long long* best, int32_t* entry, cudaStream_t s);
cudaError_t launch_knn_simt(const void* xr, int64_t m, const void* xc, int64_t n, int dtype,
                            int dpad, int Lp, int self_excl, uint64_t* rowbuf, int cpl,
                            int grid, int32_t* ids, uint32_t* thr, uint32_t* status,
                            cudaStream_t s);
// u8 (8-bit rows of the points, u8w words each) may be null; when given for rows = columns of
// exact integer data the distances come from the 8-bit rows.
cudaError_t launch_rerank(const void* xr, const void* xc, int dtype, int64_t m, int d, int dpad,
                          const int32_t* sids, const uint32_t* sthr, int Lp, int L,
                          const ScreenModel& sm, float band, int exact, int32_t* out_ids,
                          float* out_dist, int32_t* fail_rows, float* fail_bound, Counters* ctr,
                          const uint8_t* u8, int u8w, cudaStream_t s);
cudaError_t launch_rescan(const void* xr, const void* xc, int dtype, int64_t m, int64_t n, int d,
                          int dpad, int self_excl, int L, const int32_t* fail_rows,
                          const float* fail_bound, Counters* ctr, int32_t* out_ids,
                          float* out_dist, cudaStream_t s);
// half_norms: scratch of n floats for the FP16 Gram-tile prune, or null.
cudaError_t launch_prune_fwd(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* cand, const float* cdist, int L, double alpha,
                             double tau, const AlphaGrid& ag, int R, float band, int32_t* fwd,
                             int32_t* fdeg,
                             Counters* ctr, const uint8_t* u8, int u8_words, float* half_norms,
                             cudaStream_t s);
// 8-bit rows (integer data spanning <= 255): words per row for d (0: unsupported), conversion.
int u8_words(int d);
cudaError_t launch_to_u8(const void* xs, int dtype, int64_t n, int d, int dpad, float vmin, int dw,
                         uint8_t* U, cudaStream_t s);
cudaError_t launch_reverse(const int32_t* fwd, const int32_t* fdeg, int64_t n, int R,
                           int32_t* indeg, int64_t* off, int32_t* cursor, int32_t* inl,
                           int64_t* blocksums, Counters* ctr, cudaStream_t s);
// Phase-3 merge of every node whose merged set fits in shared memory; the others are
// appended to big_list (count in ctr->nbig) for launch_merge_big.  big_list holds 2 n entries
// (the second half is the 8-bit path's list between its two passes).
cudaError_t launch_merge(const void* xs, int dtype, int64_t n, int d, int dpad,
                         const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                         const int32_t* inl, double alpha, double tau, const AlphaGrid& ag,
                         int R, float band, int exact, int32_t* adj, int32_t* deg, int rs,
                         Counters* ctr, int32_t* big_list, const uint8_t* u8, int u8_words,
                         const MergeScratch& ms, cudaStream_t s);
// Merge of the listed nodes with per-CTA global scratch of 17 * big_cap bytes (grid CTAs).
cudaError_t launch_merge_big(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                             const int32_t* inl, double alpha, double tau, const AlphaGrid& ag,
                             int R, float band, int exact, int32_t* adj, int32_t* deg, int rs,
                             Counters* ctr, int32_t* big_list, int nbig, unsigned char* scratch,
                             int big_cap, int grid, cudaStream_t s);
// Phase 4 (connectivity) pieces, k_connect.cu.  counts_dev / counts_host: int[4].
cudaError_t launch_bfs(const int32_t* adj, const int32_t* deg, int Rs, int64_t n, int32_t s,
                       int32_t* reached, int32_t* fa, int32_t* fb, int* counts_dev,
                       int* counts_host, cudaStream_t st);
cudaError_t launch_collect(const int32_t* reached, int64_t n, int32_t* U, int* nu_dev,
                           cudaStream_t st);
// has_in[v] = 1 for every edge u -> v of the current rows (0 elsewhere).
cudaError_t launch_has_in(const int32_t* adj, const int32_t* deg, int Rs, int64_t n, int32_t* has_in,
                          cudaStream_t st);
// rp[i] = the first of U[i]'s kc search results whose row has a free slot, or -1; *nz_dev (zeroed
// here) = how many of them have no in-edge.
cudaError_t launch_pick(const int32_t* U, const int32_t* r, int nu, int kc, const int32_t* deg,
                        int Rs, const int32_t* has_in, int32_t* rp, int* nz_dev, cudaStream_t st);
// One claim-and-link step: every row r with a free slot named by a live rp[i] (only points
// without in-edges when zonly) gets the edge r -> (smallest such U[i]); the linked entries are
// retired (rp = -1).  best: n ints, all 0x7fffffff between calls.  *added_dev (zeroed here) =
// edges added.
cudaError_t launch_claim_link(const int32_t* U, int32_t* rp, int nu, const int32_t* has_in, int zonly,
                              int32_t* best, int32_t* adj, int32_t* deg, int Rs, int* added_dev,
                              cudaStream_t st);
cudaError_t launch_fill(int32_t* a, int64_t n, int32_t v, cudaStream_t st);

// k_beam.cu: the paper's candidate route (beam search on a K-NN graph G0)
cudaError_t launch_iota(int32_t* a, int64_t n, cudaStream_t s);
cudaError_t launch_strip_self(const int32_t* ids, const float* dists, int64_t n, int C, int32_t* cand,
                              float* cdist, uint32_t* status, cudaStream_t s);
cudaError_t launch_check_knn_graph(const int32_t* g, int64_t n, int K, uint32_t* status, cudaStream_t s);
constexpr int REPAIR_SLOTS = 8;   // adjacency row slots beyond R for phase-4 edges
constexpr int CONNECT_L = 32;     // default beam width of the phase-4 searches

int num_sms();
// True when the tensor-core Gram-tile prune (k_prune_tc.cu) takes lists of L entries with
// out-degree bound R on 8-bit rows of dw 32-bit words (U non-null).
bool gram_prune_ok(const uint8_t* U, int dw, int L, int R);
// The same for FP16 rows (dtype CNG_F16, dpad 64 or 128, fixed alpha).
bool gram_prune_f16_ok(int dtype, int dpad, int L, int R, bool adaptive);
// True when the CUDA-core all-pairs prune takes lists of L with bound R (float rows).
bool pairs_prune_ok(int L, int R, bool adaptive);
// k_entry_noalloc.cu: the navigating node using a fixed file-scope device array as scratch.
int64_t entry_noalloc_need(int64_t n, int d);      // doubles of scratch a call needs
int64_t entry_noalloc_capacity();                  // doubles the array holds
cudaError_t launch_entry_noalloc(const void* X, int dtype, int64_t n, int d, int32_t* out,
                                 cudaStream_t s);
int64_t reverse_blocksums_len(int64_t n);

}  // namespace cng
