// k_order.cu -- locality order of the point set for the tensor-core screen (an engineering
// addition; the paper has no counterpart).
//
// The screen keeps, for every row, the L' smallest screened scores seen so far; a 32-column
// chunk in which some row of a warp scores below its current threshold takes the slow append
// path.  With the columns swept in input order (random with respect to each row) the
// thresholds fall slowly and a large share of the chunks take that path.  Sorting the points
// into a k-d order, and starting each wave of row blocks at its own position in that order,
// brings most of a row's nearest columns first, so its threshold is tight early and most later
// chunks take the fast path.  The order changes nothing but speed: the screen only proposes
// candidates, and the rerank certifies them exactly (rows it cannot certify are rescanned).
//
// The order: 16 random +-1 projections of every point; then, level by level, every segment of
// the current order is sorted (stably) by the projection with the largest variance over a
// fixed sample of the segment and split at its middle position (a k-d tree with median
// splits), until segments hold at most ORD_LEAF points.  Segment bounds follow from n alone:
// a segment [a, b) has the children [a, a + (b - a) / 2) and [a + (b - a) / 2, b).  Each level
// is one stable LSD radix sort of 32-bit keys -- the segment id above the projection value
// quantised over the sample's range -- carrying the point ids.  Everything is deterministic.
#include <float.h>

#include "cng_internal.h"
#include "device_common.cuh"
#include "launch_count.h"
#include "order_internal.h"

namespace cng {

constexpr int ORD_M = 16;         // projections
constexpr int ORD_SAMPLE = 256;   // sample per segment for the split coordinate
constexpr int ORD_LEAF = 256;     // segments stop splitting at this size
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;  // keys per radix block

CNG_DEV uint32_t ord_mix(uint32_t x) {  // 32-bit finaliser of MurmurHash3
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// P[i][c] = sum_j s(j, c) x[i][j], s(j, c) = +-1 from bit c of a hash of j.  One warp per row.
template <typename T>
__global__ void __launch_bounds__(256) ord_project_kernel(const T* __restrict__ xs, int64_t n, int d,
                                                          int dpad, float* __restrict__ P) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < n; row += nw) {
    float acc[ORD_M];
#pragma unroll
    for (int c = 0; c < ORD_M; ++c) acc[c] = 0.f;
    for (int j = lane; j < d; j += 32) {
      const float v = to_f(xs[row * dpad + j]);
      const uint32_t h = ord_mix((uint32_t)j * 0x9e3779b9u + 0x7f4a7c15u);
#pragma unroll
      for (int c = 0; c < ORD_M; ++c) acc[c] += ((h >> c) & 1u) ? v : -v;
    }
#pragma unroll
    for (int c = 0; c < ORD_M; ++c)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(FULL, acc[c], o);
#pragma unroll
    for (int c = 0; c < ORD_M; ++c)
      if (lane == c) P[row * ORD_M + c] = acc[c];
  }
}

CNG_DEV void seg_bounds(int64_t n, int level, int64_t s, int64_t* a, int64_t* b) {
  int64_t lo = 0, hi = n;
  for (int i = level - 1; i >= 0; --i) {
    const int64_t mid = lo + (hi - lo) / 2;
    if ((s >> i) & 1)
      lo = mid;
    else
      hi = mid;
  }
  *a = lo;
  *b = hi;
}

CNG_DEV int64_t seg_of(int64_t n, int level, int64_t p) {
  int64_t lo = 0, hi = n, s = 0;
  for (int i = 0; i < level; ++i) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (p >= mid) {
      s = 2 * s + 1;
      lo = mid;
    } else {
      s = 2 * s;
      hi = mid;
    }
  }
  return s;
}

// One block per segment: the projection of largest variance over an evenly spaced sample of
// the segment (lowest index on ties) and that projection's sample range.
__global__ void __launch_bounds__(ORD_SAMPLE) ord_choose_kernel(const float* __restrict__ P,
                                                                const int32_t* __restrict__ perm,
                                                                int64_t n, int level,
                                                                int32_t* csel, float* clo, float* chi) {
  __shared__ float sv[ORD_SAMPLE][ORD_M + 1];
  __shared__ float var_s[ORD_M], lo_s[ORD_M], hi_s[ORD_M];
  const int t = threadIdx.x;
  int64_t a, b;
  seg_bounds(n, level, blockIdx.x, &a, &b);
  const int64_t len = b - a;
  const int cnt = (int)(len < ORD_SAMPLE ? len : ORD_SAMPLE);
  if (t < cnt) {
    const int64_t id = perm[a + (t * len) / cnt];
#pragma unroll
    for (int c = 0; c < ORD_M; ++c) sv[t][c] = P[id * ORD_M + c];
  }
  __syncthreads();
  if (t < ORD_M) {
    float mean = 0.f, lo = FLT_MAX, hi = -FLT_MAX;
    for (int i = 0; i < cnt; ++i) {
      const float v = sv[i][t];
      mean += v;
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
    mean = cnt > 0 ? mean / (float)cnt : 0.f;
    float var = 0.f;
    for (int i = 0; i < cnt; ++i) {
      const float e = sv[i][t] - mean;
      var = fmaf(e, e, var);
    }
    var_s[t] = var;
    lo_s[t] = cnt > 0 ? lo : 0.f;
    hi_s[t] = cnt > 0 ? hi : 0.f;
  }
  __syncthreads();
  if (t == 0) {
    int best = 0;
    for (int c = 1; c < ORD_M; ++c)
      if (var_s[c] > var_s[best]) best = c;
    csel[blockIdx.x] = best;
    clo[blockIdx.x] = lo_s[best];
    chi[blockIdx.x] = hi_s[best];
  }
}

// key = segment id in the top `level` bits, the chosen projection quantised over the sample
// range in the remaining 32 - level bits (values outside the range clamp to its ends).
__global__ void ord_key_kernel(const float* __restrict__ P, const int32_t* __restrict__ perm,
                               int64_t n, int level, const int32_t* __restrict__ csel,
                               const float* __restrict__ clo, const float* __restrict__ chi,
                               uint32_t* __restrict__ key) {
  const int vb = 32 - level;
  const double qmax = (double)((1ull << vb) - 1);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = seg_of(n, level, p);
    const float v = P[(int64_t)perm[p] * ORD_M + csel[s]];
    const double lo = clo[s], hi = chi[s];
    double f = hi > lo ? ((double)v - lo) / (hi - lo) : 0.5;
    f = fmin(fmax(f, 0.0), 1.0);
    const uint64_t q = (uint64_t)(f * qmax);
    key[p] = (uint32_t)(((uint64_t)s << vb) | q);
  }
}

// ---- stable LSD radix sort, 8-bit digits ------------------------------------------------------
__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(const uint32_t* __restrict__ key,
                                                             int64_t n, int shift, int nblk,
                                                             uint32_t* __restrict__ ghist) {
  __shared__ uint32_t h[256];
  const int t = threadIdx.x;
  h[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + t;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  ghist[(int64_t)t * nblk + blockIdx.x] = h[t];  // digit-major
}

// Exclusive scan in place of len counts (one block of 1024 threads).
__global__ void __launch_bounds__(1024) rs_scan_kernel(uint32_t* __restrict__ g, int64_t len) {
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (len + 1023) / 1024;
  const int64_t a = min(len, t * per), b = min(len, a + per);
  uint32_t s = 0;
  for (int64_t i = a; i < b; ++i) s += g[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;
  for (int64_t i = a; i < b; ++i) {
    const uint32_t c = g[i];
    g[i] = run;
    run += c;
  }
}

// Stable scatter: the block's keys in rounds of 256 consecutive positions; within a round the
// rank of a key among equal digits is its warp rank plus the counts of earlier warps.
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t n, int shift, int nblk, const uint32_t* __restrict__ gscan) {
  constexpr int NW = RS_THREADS / 32;
  __shared__ uint32_t wc[NW][256];
  __shared__ uint32_t run[256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  run[t] = gscan[(int64_t)t * nblk + blockIdx.x];
  uint32_t my_tot = 0;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
#pragma unroll
    for (int w = 0; w < NW; ++w) wc[w][t] = 0;
    if (r > 0) run[t] += my_tot;
    __syncthreads();
    const int64_t i = base + r * RS_THREADS + t;
    const bool valid = i < n;
    const uint32_t k = valid ? kin[i] : 0u;
    const uint32_t dg = valid ? (k >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(FULL, dg);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wc[warp][dg] = __popc(peers);
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t c = wc[w][t];
      wc[w][t] = s;
      s += c;
    }
    my_tot = s;
    __syncthreads();
    if (valid) {
      const uint32_t pos = run[dg] + wc[warp][dg] + rank;
      kout[pos] = k;
      vout[pos] = vin[i];
    }
    __syncthreads();
  }
}

__global__ void ord_iota_kernel(int32_t* perm, int64_t n) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x)
    perm[p] = (int32_t)p;
}

// xo[p] = xi[perm[p]] (rows of kpad 16-bit values), nbo[p] = nbi[perm[p]].  One warp per row.
__global__ void __launch_bounds__(256) ord_gather_kernel(const uint4* __restrict__ xi,
                                                         const float* __restrict__ nbi,
                                                         const int32_t* __restrict__ perm, int64_t n,
                                                         int row_vecs, uint4* __restrict__ xo,
                                                         float* __restrict__ nbo) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = w0; p < n; p += nw) {
    const int64_t src = perm[p];
    for (int v = lane; v < row_vecs; v += 32) xo[p * row_vecs + v] = xi[src * row_vecs + v];
    if (lane == 0) nbo[p] = nbi[src];
  }
}

int order_levels(int64_t n) {
  int levels = 0;
  while ((n >> levels) > ORD_LEAF && levels < 24) ++levels;
  return levels;
}

size_t order_scratch_bytes(int64_t n) {
  const int levels = order_levels(n);
  const int64_t nseg = levels > 0 ? (int64_t)1 << (levels - 1) : 1;
  const int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) & ~size_t(255); };
  add((size_t)n * ORD_M * 4);            // projections
  add((size_t)n * 4);                    // perm (second buffer)
  add((size_t)n * 4);                    // keys
  add((size_t)n * 4);                    // keys (second buffer)
  add((size_t)nseg * 12);                // csel, clo, chi
  add((size_t)256 * nblk * 4);           // digit counts
  return b;
}

static cudaError_t radix_sort(uint32_t* k0, int32_t* v0, uint32_t* k1, int32_t* v1, int64_t n,
                              uint32_t* ghist, cudaStream_t s) {
  const int nblk = (int)((n + RS_TILE - 1) / RS_TILE);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = pass * 8;
    uint32_t* ki = (pass & 1) ? k1 : k0;
    int32_t* vi = (pass & 1) ? v1 : v0;
    uint32_t* ko = (pass & 1) ? k0 : k1;
    int32_t* vo = (pass & 1) ? v0 : v1;
    count_launch();
    rs_hist_kernel<<<nblk, RS_THREADS, 0, s>>>(ki, n, shift, nblk, ghist);
    count_launch();
    rs_scan_kernel<<<1, 1024, 0, s>>>(ghist, (int64_t)256 * nblk);
    count_launch();
    rs_scatter_kernel<<<nblk, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, nblk, ghist);
  }
  return cudaGetLastError();  // four passes: the result is back in (k0, v0)
}

cudaError_t launch_order(const void* xs, int dtype, int64_t n, int d, int dpad, int32_t* perm,
                         void* scratch, cudaStream_t s) {
  const int levels = order_levels(n);
  const int64_t nseg = levels > 0 ? (int64_t)1 << (levels - 1) : 1;
  const int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
  unsigned char* p = static_cast<unsigned char*>(scratch);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  float* P = static_cast<float*>(take((size_t)n * ORD_M * 4));
  int32_t* perm2 = static_cast<int32_t*>(take((size_t)n * 4));
  uint32_t* key0 = static_cast<uint32_t*>(take((size_t)n * 4));
  uint32_t* key1 = static_cast<uint32_t*>(take((size_t)n * 4));
  unsigned char* segv = static_cast<unsigned char*>(take((size_t)nseg * 12));
  int32_t* csel = reinterpret_cast<int32_t*>(segv);
  float* clo = reinterpret_cast<float*>(segv + nseg * 4);
  float* chi = reinterpret_cast<float*>(segv + nseg * 8);
  uint32_t* ghist = static_cast<uint32_t*>(take((size_t)256 * nblk * 4));

  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 16);
  count_launch();
  ord_iota_kernel<<<grid, 256, 0, s>>>(perm, n);
  const int pgrid = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  count_launch();
  if (dtype == CNG_F32)
    ord_project_kernel<float><<<pgrid, 256, 0, s>>>((const float*)xs, n, d, dpad, P);
  else
    ord_project_kernel<__half><<<pgrid, 256, 0, s>>>((const __half*)xs, n, d, dpad, P);
  for (int level = 0; level < levels; ++level) {
    count_launch();
    ord_choose_kernel<<<(unsigned)((int64_t)1 << level), ORD_SAMPLE, 0, s>>>(P, perm, n, level, csel,
                                                                             clo, chi);
    count_launch();
    ord_key_kernel<<<grid, 256, 0, s>>>(P, perm, n, level, csel, clo, chi, key0);
    cudaError_t e = radix_sort(key0, perm, key1, perm2, n, ghist, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_order_gather(const void* xi, const float* nbi, const int32_t* perm, int64_t n,
                                int kpad, void* xo, float* nbo, cudaStream_t s) {
  const int row_vecs = kpad * 2 / 16;
  const int grid = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  count_launch();
  ord_gather_kernel<<<grid, 256, 0, s>>>(static_cast<const uint4*>(xi), nbi, perm, n, row_vecs,
                                         static_cast<uint4*>(xo), nbo);
  return cudaGetLastError();
}

}  // namespace cng
