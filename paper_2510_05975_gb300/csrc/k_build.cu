// k_build.cu -- candidate-list kernels of the alpha-CNG build (sm_103a):
//   K0 prep      padded storage copy, tensor-core operand copy, norms, exactness statistics
//   K3 entry     navigating node: blocked FP64 centroid and exact (D, id) argmin
//                (Alg. 3 phase 1, exact form)
//   K1f screen   FP32 CUDA-core distance tiles with a fused per-row top-L' buffer
//   K2 rerank    FP32 recompute of the screened ids, (d, id) sort, certification of the
//                screen, FP64 re-decision of near-tied neighbours in the order
//   rescan       exact fallback for rows the certification rejects
// The candidate list of p is the L points u != p with the smallest (D(p,u), id(u)) -- the
// exact form of Alg. 3 phase 2's candidate set.
#include <float.h>

#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"

namespace cng {

// ============================================================================================
// K0: preparation
// ============================================================================================
template <typename Tin, typename Tst>
__global__ void __launch_bounds__(256) prep_kernel(const Tin* __restrict__ P, int64_t n, int d,
                                                   int dpad, Tst* __restrict__ xs,
                                                   __nv_bfloat16* __restrict__ xb_bf,
                                                   __half* __restrict__ xb_h, int kpad,
                                                   float* __restrict__ nb, float* __restrict__ rb,
                                                   float scale, PrepStats* st) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool screen = xb_bf != nullptr || xb_h != nullptr;
  const int width = max(dpad, screen ? kpad : 0);
  bool nonint = false;
  float vmin = FLT_MAX, vmax = -FLT_MAX, nbmax = 0.f, rbmax = 0.f, normmax = 0.f, unitdev = 0.f;
  for (int64_t row = gw; row < n; row += nw) {
    float ssq = 0.f, snb = 0.f, srb = 0.f;
    for (int c = lane; c < width; c += 32) {
      float v = c < d ? to_f(P[row * d + c]) : 0.f;
      if (c < dpad) xs[row * dpad + c] = (Tst)v;
      if (screen && c < kpad) {
        float fb;
        const float vs = v * scale;  // exact: scale is a power of two
        if (xb_bf) {
          __nv_bfloat16 b = __float2bfloat16_rn(vs);
          xb_bf[row * kpad + c] = b;
          fb = __bfloat162float(b);
        } else {
          __half h = __float2half_rn(vs);
          xb_h[row * kpad + c] = h;
          fb = __half2float(h);
        }
        snb = fmaf(fb, fb, snb);
        float e = fb - vs;
        srb = fmaf(e, e, srb);
      }
      if (c < d) {
        ssq = fmaf(v, v, ssq);
        nonint |= (v != rintf(v));
        vmin = fminf(vmin, v);
        vmax = fmaxf(vmax, v);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ssq += __shfl_xor_sync(FULL, ssq, o);
      snb += __shfl_xor_sync(FULL, snb, o);
      srb += __shfl_xor_sync(FULL, srb, o);
    }
    if (screen && lane == 0) {
      nb[row] = snb;
      rb[row] = srb > 0.f ? sqrtf(srb) * (1.f + 1e-6f) : 0.f;
    }
    float nrm = sqrtf(ssq);
    nbmax = fmaxf(nbmax, snb);
    rbmax = fmaxf(rbmax, srb > 0.f ? sqrtf(srb) * (1.f + 1e-6f) : 0.f);
    normmax = fmaxf(normmax, nrm);
    unitdev = fmaxf(unitdev, fabsf(nrm - 1.f));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vmin = fminf(vmin, __shfl_xor_sync(FULL, vmin, o));
    vmax = fmaxf(vmax, __shfl_xor_sync(FULL, vmax, o));
  }
  unsigned ni = __ballot_sync(FULL, nonint);
  if (lane == 0 && gw < n) {
    if (ni) atomicOr(&st->nonint, 1u);
    atomicMin(&st->vmin_key, fkey(vmin));
    atomicMax(&st->vmax_key, fkey(vmax));
    atomicMax(&st->nbmax_bits, __float_as_uint(nbmax));
    atomicMax(&st->rbmax_bits, __float_as_uint(rbmax));
    atomicMax(&st->normmax_bits, __float_as_uint(normmax));
    atomicMax(&st->unitdev_bits, __float_as_uint(unitdev));
  }
}

cudaError_t launch_prep(const void* pts, int dtype, int64_t n, int d, int dpad, void* xs,
                        __nv_bfloat16* xb_bf, __half* xb_h, int kpad, float* nb, float* rb,
                        float scale, PrepStats* st, cudaStream_t s) {
  int64_t warps = (n + 3) / 4;
  int grid = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)num_sms() * 16);
  if (grid < 1) grid = 1;
  count_launch();
  if (dtype == CNG_F32)
    prep_kernel<float, float><<<grid, 256, 0, s>>>((const float*)pts, n, d, dpad, (float*)xs,
                                                   xb_bf, xb_h, kpad, nb, rb, scale, st);
  else
    prep_kernel<__half, __half><<<grid, 256, 0, s>>>((const __half*)pts, n, d, dpad,
                                                     (__half*)xs, xb_bf, xb_h, kpad, nb, rb, scale,
                                                     st);
  return cudaGetLastError();
}

// max |x| (float bits) and whether some coordinate is not an integer, over an unpadded n x d
// matrix: out[0], out[1] (out zeroed by the caller).
template <typename T>
__global__ void absmax_kernel(const T* __restrict__ P, int64_t total, uint32_t* out) {
  float m = 0.f;
  bool nonint = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = to_f(P[e]);
    m = fmaxf(m, fabsf(v));
    nonint |= v != rintf(v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
  const unsigned ni = __ballot_sync(FULL, nonint);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], __float_as_uint(m));
    if (ni) atomicOr(&out[1], 1u);
  }
}

cudaError_t launch_absmax(const void* pts, int dtype, int64_t n, int d, uint32_t* out,
                          cudaStream_t s) {
  const int64_t total = n * (int64_t)d;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8));
  count_launch();
  if (dtype == CNG_F32)
    absmax_kernel<float><<<grid, 256, 0, s>>>((const float*)pts, total, out);
  else
    absmax_kernel<__half><<<grid, 256, 0, s>>>((const __half*)pts, total, out);
  return cudaGetLastError();
}

// ============================================================================================
// K3: navigating node
// ============================================================================================
constexpr int CENTROID_BLOCK = 4096;  // rows per block sum; same order as the definition

template <typename T>
__global__ void centroid_part_kernel(const T* __restrict__ xs, int64_t n, int d, int dpad,
                                     double* __restrict__ part) {
  int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= d) return;
  int64_t b0 = (int64_t)blockIdx.x * CENTROID_BLOCK;
  int64_t e = min(n, b0 + CENTROID_BLOCK);
  double s = 0.0;
  for (int64_t i = b0; i < e; ++i) s = __dadd_rn(s, (double)to_f(xs[i * dpad + j]));
  part[(int64_t)blockIdx.x * d + j] = s;
}

__global__ void centroid_final_kernel(const double* __restrict__ part, int nblk, int64_t n, int d,
                                      double* __restrict__ cen, unsigned long long* best) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) { best[0] = ~0ull; best[1] = ~0ull; }
  if (j >= d) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t = __dadd_rn(t, part[(int64_t)b * d + j]);
  cen[j] = __ddiv_rn(t, (double)n);
}

// D(c, x_i) canonical; min over i of the double's bits (>= 0, so bit order = value order).
template <typename T>
__global__ void __launch_bounds__(256) entry_dist_kernel(const T* __restrict__ xs, int64_t n, int d,
                                                         int dpad, const double* __restrict__ cen,
                                                         unsigned long long* __restrict__ dbits,
                                                         unsigned long long* best) {
  extern __shared__ double cs[];
  for (int j = threadIdx.x; j < d; j += blockDim.x) cs[j] = cen[j];
  __syncthreads();
  unsigned long long mine = ~0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T* x = xs + i * dpad;
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      double t = __dsub_rn(cs[j], (double)to_f(x[j]));
      s = __dadd_rn(s, __dmul_rn(t, t));
    }
    unsigned long long b = (unsigned long long)__double_as_longlong(__dsqrt_rn(s));
    dbits[i] = b;
    mine = min(mine, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(FULL, mine, o));
  if ((threadIdx.x & 31) == 0 && mine != ~0ull) atomicMin(&best[0], mine);
}

__global__ void entry_pick_kernel(const unsigned long long* __restrict__ dbits, int64_t n,
                                  unsigned long long* best) {
  unsigned long long m = best[0];
  unsigned long long mine = ~0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (dbits[i] == m) mine = min(mine, (unsigned long long)i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(FULL, mine, o));
  if ((threadIdx.x & 31) == 0 && mine != ~0ull) atomicMin(&best[1], mine);
}

__global__ void entry_write_kernel(const unsigned long long* best, int32_t* entry) {
  *entry = (int32_t)best[1];
}

cudaError_t launch_entry(const void* xs, int dtype, int64_t n, int d, int dpad, double* part,
                         double* cen, unsigned long long* best, int32_t* entry, cudaStream_t s) {
  int nblk = (int)((n + CENTROID_BLOCK - 1) / CENTROID_BLOCK);
  dim3 g1(nblk, (d + 127) / 128);
  // `part` holds nblk * d doubles followed by n words of distance bits
  unsigned long long* dbits = reinterpret_cast<unsigned long long*>(part + (int64_t)nblk * d);
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  if (dtype == CNG_F32) {
    count_launch();
    centroid_part_kernel<float><<<g1, 128, 0, s>>>((const float*)xs, n, d, dpad, part);
    count_launch();
    centroid_final_kernel<<<(d + 127) / 128, 128, 0, s>>>(part, nblk, n, d, cen, best);
    count_launch();
    entry_dist_kernel<float><<<grid, 256, d * sizeof(double), s>>>((const float*)xs, n, d, dpad,
                                                                   cen, dbits, best);
  } else {
    count_launch();
    centroid_part_kernel<__half><<<g1, 128, 0, s>>>((const __half*)xs, n, d, dpad, part);
    count_launch();
    centroid_final_kernel<<<(d + 127) / 128, 128, 0, s>>>(part, nblk, n, d, cen, best);
    count_launch();
    entry_dist_kernel<__half><<<grid, 256, d * sizeof(double), s>>>((const __half*)xs, n, d,
                                                                    dpad, cen, dbits, best);
  }
  count_launch();
  entry_pick_kernel<<<grid, 256, 0, s>>>(dbits, n, best);
  count_launch();
  entry_write_kernel<<<1, 1, 0, s>>>(best, entry);
  return cudaGetLastError();
}

// ============================================================================================
// K1f: FP32 CUDA-core screen with fused top-L' selection
// ============================================================================================
// CTA tile 128 rows x 128 columns, 256 threads, 8 x 8 register micro-tile per thread, direct
// squared differences.  Each CTA owns 128 row buffers (global, `cap` entries each) for the
// whole column sweep of its row block; an entry is appended only if its key is below the
// row's threshold; a buffer that could overflow on the next tile is compacted to its Lp
// smallest entries by one warp (radix select), which lowers the threshold.
constexpr int FB = 128;
constexpr int FK = 16;
constexpr int FPAD = 4;

CNG_DEV void load8(const float* __restrict__ base, int64_t row, int dpad, int k, float* v) {
  if (row < 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.f;
    return;
  }
  const float4* p = reinterpret_cast<const float4*>(base + row * dpad + k);
  float4 a = __ldg(p), b = __ldg(p + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
CNG_DEV void load8(const __half* __restrict__ base, int64_t row, int dpad, int k, float* v) {
  if (row < 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.f;
    return;
  }
  uint4 u = __ldg(reinterpret_cast<const uint4*>(base + row * dpad + k));
  float4 a = h8lo(u), b = h8hi(u);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

template <typename T, int CPL>
__global__ void __launch_bounds__(256, 2)
knn_simt_kernel(const T* __restrict__ Xr, int64_t m, const T* __restrict__ Xc, int64_t n, int dpad,
                int Lp, int self_excl, uint64_t* __restrict__ rowbuf, int32_t* __restrict__ out_ids,
                uint32_t* __restrict__ out_thr, uint32_t* __restrict__ status) {
  __shared__ __align__(16) float As[FK][FB + FPAD];
  __shared__ __align__(16) float Bs[FK][FB + FPAD];
  __shared__ uint32_t thr[FB];
  __shared__ int cnt[FB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tx = tid & 15, ty = tid >> 4;
  constexpr int cap = CPL * 32;
  uint64_t* myrb = rowbuf + (size_t)blockIdx.x * FB * cap;
  const int64_t nrb = (m + FB - 1) / FB;
  for (int64_t rbk = blockIdx.x; rbk < nrb; rbk += gridDim.x) {
    const int64_t r0 = rbk * FB;
    if (tid < FB) { thr[tid] = 0xffffffffu; cnt[tid] = 0; }
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += FB) {
      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      for (int k0 = 0; k0 < dpad; k0 += FK) {
        {
          const int r = tid >> 1, kk = (tid & 1) * 8;
          float v[8];
          const int64_t gr = r0 + r, gc = c0 + r;
          load8(Xr, gr < m ? gr : -1, dpad, k0 + kk, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) As[kk + j][r] = v[j];
          load8(Xc, gc < n ? gc : -1, dpad, k0 + kk, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) Bs[kk + j][r] = v[j];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < FK; ++kk) {
          float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
          float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
          float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
          float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
          const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float t = a[i] - b[j];
              acc[i][j] = fmaf(t, t, acc[i][j]);
            }
        }
        __syncthreads();
      }
      // fused selection: append entries below the row threshold
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = ty * 8 + i;
        const int64_t grow = r0 + row;
        if (grow >= m) continue;
        const uint32_t th = thr[row];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int64_t col = c0 + tx * 8 + j;
          const uint32_t k = fkey(acc[i][j]);
          if (col < n && k < th && !(self_excl && col == grow)) {
            int slot = atomicAdd(&cnt[row], 1);
            if (slot < cap)
              myrb[(size_t)row * cap + slot] = ((uint64_t)k << 32) | (uint32_t)col;
            else
              set_status(status, ST_OVERFLOW);
          }
        }
      }
      __syncthreads();
      for (int row = warp; row < FB; row += 8) {
        int c = min(cnt[row], cap);
        if (c > cap - FB) {
          uint32_t k = warp_compact<CPL>(myrb + (size_t)row * cap, c, Lp, lane);
          if (lane == 0) { thr[row] = k; cnt[row] = Lp; }
        }
      }
      __syncthreads();
    }
    for (int row = warp; row < FB; row += 8) {
      const int64_t grow = r0 + row;
      if (grow >= m) continue;
      int c = min(cnt[row], cap);
      uint32_t th = thr[row];
      if (c > Lp) {
        th = warp_compact<CPL>(myrb + (size_t)row * cap, c, Lp, lane);
        c = Lp;
      }
      for (int t = lane; t < Lp; t += 32)
        out_ids[grow * Lp + t] = t < c ? key_id(myrb[(size_t)row * cap + t]) : -1;
      if (lane == 0) out_thr[grow] = th;
    }
    __syncthreads();
  }
}

template <typename T, int CPL>
static cudaError_t knn_simt_t(const void* xr, int64_t m, const void* xc, int64_t n, int dpad,
                              int Lp, int self_excl, uint64_t* rowbuf, int grid, int32_t* ids,
                              uint32_t* thr, uint32_t* status, cudaStream_t s) {
  count_launch();
  knn_simt_kernel<T, CPL><<<grid, 256, 0, s>>>((const T*)xr, m, (const T*)xc, n, dpad, Lp,
                                               self_excl, rowbuf, ids, thr, status);
  return cudaGetLastError();
}

// cpl = buffer capacity / 32; capacity must exceed Lp + 128 (one tile of appends).
cudaError_t launch_knn_simt(const void* xr, int64_t m, const void* xc, int64_t n, int dtype,
                            int dpad, int Lp, int self_excl, uint64_t* rowbuf, int cpl,
                            int grid, int32_t* ids, uint32_t* thr, uint32_t* status,
                            cudaStream_t s) {
#define CNG_KS(C)                                                                              \
  case C:                                                                                      \
    return dtype == CNG_F32                                                                    \
               ? knn_simt_t<float, C>(xr, m, xc, n, dpad, Lp, self_excl, rowbuf, grid, ids,    \
                                      thr, status, s)                                          \
               : knn_simt_t<__half, C>(xr, m, xc, n, dpad, Lp, self_excl, rowbuf, grid, ids,   \
                                       thr, status, s);
  switch (cpl) {
    CNG_KS(8)
    CNG_KS(12)
    CNG_KS(16)
    CNG_KS(20)
    default:
      return cudaErrorInvalidValue;
  }
#undef CNG_KS
}

// ============================================================================================
// K2: rerank, certify, order near-ties
// ============================================================================================
constexpr int RR_WARPS = 4;
constexpr int RR_P2 = 512;      // max screened list (power of two)
constexpr int RR_RUN = 256;     // longest near-tie run re-sorted in FP64
constexpr int RR_G = 8;         // lanes per distance

CNG_DEV void warp_bitonic(uint64_t* a, int P2, int lane) {
  for (int k = 2; k <= P2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P2; i += 32) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) { a[i] = y; a[ixj] = x; }
        }
      }
      __syncwarp();
    }
}

// Re-sort, by the canonical (D, id) order, every run of neighbours in keys[0..cnt) whose FP32
// squared distances are pairwise near-tied and that starts before position `upto`.  `row` is
// the stored row vector (exact values).  Runs are gathered in batches (up to 32 runs, RR_RUN
// members); the canonical distances of a batch's members are computed in parallel, one per
// lane, then lane 0 insertion-sorts each run.  rdesc: [3][32] ints of warp scratch (run start,
// length, offset in d64).  Returns the number of runs re-decided.
template <typename T>
CNG_DEV int fix_runs_warp(uint64_t* keys, int cnt, int upto, const T* __restrict__ row,
                          const T* __restrict__ Xc, int dpad, int d, float band, double* d64,
                          int* rdesc, int lane, uint32_t* status) {
  int runs = 0;
  int i = 0;
  while (i < upto && i + 1 < cnt) {
    int nb = 0, total = 0;
    while (nb < 32 && i < upto && i + 1 < cnt) {
      // the next run start >= i (lane-parallel scan, 32 pairs at a time)
      int s = -1;
      for (int b = i; b < upto && b + 1 < cnt && s < 0; b += 32) {
        int t = b + lane;
        bool nt = t < upto && t + 1 < cnt && near_tie(key_dist(keys[t]), key_dist(keys[t + 1]), band);
        unsigned bal = __ballot_sync(FULL, nt);
        if (bal) s = b + __ffs(bal) - 1;
      }
      if (s < 0) {
        i = upto;
        break;
      }
      int e = s + 1;  // run is [s, e]
      while (e + 1 < cnt && near_tie(key_dist(keys[e]), key_dist(keys[e + 1]), band)) ++e;
      int len = e - s + 1;
      if (len > RR_RUN) {
        if (lane == 0) set_status(status, ST_OVF_RUN);
        len = RR_RUN;
        e = s + len - 1;
      }
      if (total + len > RR_RUN) break;  // this run opens the next batch
      if (lane == 0) {
        rdesc[nb] = s;
        rdesc[32 + nb] = len;
        rdesc[64 + nb] = total;
      }
      total += len;
      ++nb;
      i = e + 1;
    }
    if (nb == 0) break;
    __syncwarp();
    for (int m = lane; m < total; m += 32) {
      int k = 0;
      while (k + 1 < nb && rdesc[64 + k + 1] <= m) ++k;
      const int pos = rdesc[k] + (m - rdesc[64 + k]);
      d64[m] = canon_dist(row, Xc + (int64_t)key_id(keys[pos]) * dpad, d);
    }
    __syncwarp();
    if (lane == 0) {  // insertion sort of each run by (d64, id)
      for (int k = 0; k < nb; ++k) {
        const int s = rdesc[k], len = rdesc[32 + k];
        double* dd = d64 + rdesc[64 + k];
        for (int a = 1; a < len; ++a) {
          double dv = dd[a];
          uint64_t kv = keys[s + a];
          int b = a - 1;
          while (b >= 0 && (dd[b] > dv || (dd[b] == dv && key_id(keys[s + b]) > key_id(kv)))) {
            dd[b + 1] = dd[b];
            keys[s + b + 1] = keys[s + b];
            --b;
          }
          dd[b + 1] = dv;
          keys[s + b + 1] = kv;
        }
      }
    }
    __syncwarp();
    runs += nb;
  }
  return runs;
}

// Squared FP32 distances of the query slice held in registers (lane l holds float4 chunks
// l, l + 32, ..., NQ of them) to two stored rows read by the whole warp (coalesced 16-byte
// loads), for rows wider than 256: two candidates per call keep 2 NQ loads in flight per lane.
// Each lane sums its chunks in order with 2 accumulators (chain <= 2 NQ elements), then a
// 5-level shuffle tree.
template <int NQ>
CNG_DEV void wide_sqdist2(const float4 (&qr)[NQ], const float* __restrict__ y0,
                          const float* __restrict__ y1, int nch, int lane, float& r0, float& r1) {
  const float4* a4 = reinterpret_cast<const float4*>(y0);
  const float4* b4 = reinterpret_cast<const float4*>(y1);
  float4 va[NQ], vb[NQ];
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const int c = lane + 32 * j;
    va[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    vb[j] = va[j];
    if (c < nch) {
      if (y0) va[j] = __ldg(a4 + c);
      if (y1) vb[j] = __ldg(b4 + c);
    }
  }
  float s0 = 0.f, s1 = 0.f, t0 = 0.f, t1 = 0.f;
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const int c = lane + 32 * j;
    if (c < nch) {
      if (j & 1) {
        acc4(qr[j], va[j], s1);
        acc4(qr[j], vb[j], t1);
      } else {
        acc4(qr[j], va[j], s0);
        acc4(qr[j], vb[j], t0);
      }
    }
  }
  float a = s0 + s1, b = t0 + t1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(FULL, a, o);
    b += __shfl_xor_sync(FULL, b, o);
  }
  r0 = a;
  r1 = b;
}

// Sorts a row's keys [0, Lp) (FP32 D^2, id), then certifies the list: every unscreened point
// is provably farther than the L-th candidate.  Rows that fail are queued for the exact rescan
// (returns false, uniform over the warp).
CNG_DEV bool rerank_sort_certify(uint64_t* keys, int P2, int cnt, int64_t row, int Lp, int L,
                                 const uint32_t* __restrict__ sthr, const ScreenModel& sm,
                                 float band, int exact, int32_t* fail_rows, float* fail_bound,
                                 Counters* ctr, int lane) {
  for (int t = Lp + lane; t < P2; t += 32) keys[t] = ~0ull;
  __syncwarp();
  warp_bitonic(keys, P2, lane);
  bool ok = true;
  const uint32_t th = sthr[row];
  if (th != 0xffffffffu && cnt >= L) {
    const float dL = key_dist(keys[L - 1]);
    const float sc = fkey_inv(th);
    if (sm.kind == 0) {
      float lb = sc * (1.f - sm.rel_err);
      ok = exact ? (sc > dL) : (lb > dL * (1.f + 2.f * band));
    } else {
      // scores are in units of scale^2 (operands scale * x, scale a power of two): compare
      // with dL scaled exactly
      const float nx = sm.nb[row];
      const float dLs = dL * sm.scale2;
      if (exact) {
        ok = (sc + nx) > dLs;
      } else {
        float nrm = sqrtf(fmaxf(nx, 0.f));
        float eacc = sm.acc_err * (nrm + sm.normmax) * (nrm + sm.normmax);
        float db = sqrtf(fmaxf(sc + nx - eacc, 0.f)) - (sm.rb[row] + sm.rbmax);
        ok = db > 0.f && db * db > dLs * (1.f + 2.f * band);
      }
    }
  }
  if (cnt < L) ok = false;
  if (!ok && lane == 0) {
    int slot = atomicAdd(&ctr->nfail, 1);
    fail_rows[slot] = (int32_t)row;
    fail_bound[slot] = cnt >= L ? key_dist(keys[L - 1]) * (1.f + 4.f * band) : INFINITY;
  }
  return ok;
}

CNG_DEV void rerank_write(const uint64_t* keys, int64_t row, int L, int32_t* __restrict__ out_ids,
                          float* __restrict__ out_dist, int lane) {
  for (int t = lane; t < L; t += 32) {
    uint64_t k = keys[t];
    out_ids[row * L + t] = key_id(k);
    out_dist[row * L + t] = sqrtf(key_dist(k));
  }
  __syncwarp();
}

template <typename T, int NQ>
__global__ void __launch_bounds__(RR_WARPS * 32)
rerank_kernel(const T* __restrict__ Xr, const T* __restrict__ Xc, int64_t m, int d, int dpad,
              const int32_t* __restrict__ sids, const uint32_t* __restrict__ sthr, int Lp, int L,
              ScreenModel sm, float band, int exact, int32_t* __restrict__ out_ids,
              float* __restrict__ out_dist, int32_t* __restrict__ fail_rows,
              float* __restrict__ fail_bound, Counters* ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P2 = Lp <= 64 ? 64 : (Lp <= 128 ? 128 : (Lp <= 256 ? 256 : 512));
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem) + warp * RR_P2;
  double* d64 = reinterpret_cast<double*>(smem + RR_WARPS * RR_P2 * 8) + warp * RR_RUN;
  int* rdesc = reinterpret_cast<int*>(smem + RR_WARPS * (RR_P2 * 8 + RR_RUN * 8)) + warp * 96;
  float* q = reinterpret_cast<float*>(smem + RR_WARPS * (RR_P2 * 8 + RR_RUN * 8 + 96 * 4)) + warp * dpad;
  const int g = lane % RR_G, grp = lane / RR_G;
  unsigned long long ties = 0;
  float err_max = 0.f;
  for (int64_t row = blockIdx.x * (int64_t)RR_WARPS + warp; row < m;
       row += (int64_t)gridDim.x * RR_WARPS) {
    const int32_t* ids = sids + row * Lp;
    int cnt = 0;
    if constexpr (NQ > 0) {
      // wide rows: the query slice in registers, one candidate per warp, two at a time
      const int nch = dpad >> 2;
      const float4* x4 = reinterpret_cast<const float4*>(Xr + row * dpad);
      float4 qr[NQ];
#pragma unroll
      for (int j = 0; j < NQ; ++j)
        qr[j] = lane + 32 * j < nch ? __ldg(x4 + lane + 32 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int t = 0; t < Lp; t += 2) {
        const int32_t i0 = ids[t], i1 = t + 1 < Lp ? ids[t + 1] : -1;
        float s0, s1;
        wide_sqdist2<NQ>(qr, i0 >= 0 ? reinterpret_cast<const float*>(Xc + (int64_t)i0 * dpad) : nullptr,
                         i1 >= 0 ? reinterpret_cast<const float*>(Xc + (int64_t)i1 * dpad) : nullptr, nch,
                         lane, s0, s1);
        if (lane == 0) {
          keys[t] = i0 >= 0 ? pack_key(s0, i0) : ~0ull;
          if (t + 1 < Lp) keys[t + 1] = i1 >= 0 ? pack_key(s1, i1) : ~0ull;
        }
        cnt += (i0 >= 0) + (t + 1 < Lp && i1 >= 0);
      }
    } else {
      load_row(q, Xr + row * dpad, dpad, lane, 32);
      __syncwarp();
      for (int t0 = 0; t0 < Lp; t0 += 32 / RR_G) {
        int t = t0 + grp;
        int32_t id = t < Lp ? ids[t] : -1;
        float s = 0.f;
        if (id >= 0) s = part_sqdist<RR_G>(q, Xc + (int64_t)id * dpad, dpad, g);
        s = group_reduce<RR_G>(s);
        if (g == 0 && t < Lp) keys[t] = id >= 0 ? pack_key(s, id) : ~0ull;
        unsigned v = __ballot_sync(FULL, g == 0 && t < Lp && id >= 0);
        cnt += __popc(v);
      }
    }
    if (!rerank_sort_certify(keys, P2, cnt, row, Lp, L, sthr, sm, band, exact, fail_rows, fail_bound,
                             ctr, lane))
      continue;
    if (!exact) ties += fix_runs_warp(keys, cnt, L, Xr + row * dpad, Xc, dpad, d, band, d64, rdesc, lane,
                                      &ctr->status);
    rerank_write(keys, row, L, out_ids, out_dist, lane);
  }
  if (lane == 0 && ties) atomicAdd(&ctr->order_ties, ties);
  (void)err_max;
}

// 8-bit rows (integer data spanning <= 255, rows and columns the same points): D^2 as the exact
// integer sum of dp4a(|u - v|, |u - v|) over 16-byte chunks, 8 lanes per candidate (one
// coalesced 128-byte row read per group) -- the value the FP32 difference form gives for such
// data, from a quarter of the bytes.  (One candidate per lane with the whole row per lane was
// slower: 11.2 against 9.0 ms at 1M x 128.)
template <int DW>
__global__ void __launch_bounds__(RR_WARPS * 32)
rerank_u8_kernel(const uint8_t* __restrict__ U, int64_t m, const int32_t* __restrict__ sids,
                 const uint32_t* __restrict__ sthr, int Lp, int L, ScreenModel sm, float band,
                 int32_t* __restrict__ out_ids, float* __restrict__ out_dist,
                 int32_t* __restrict__ fail_rows, float* __restrict__ fail_bound, Counters* ctr) {
  constexpr int NC = DW / 4;  // 16-byte chunks per row, <= RR_G
  static_assert(NC <= RR_G, "one chunk per lane of a group");
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P2 = Lp <= 64 ? 64 : (Lp <= 128 ? 128 : (Lp <= 256 ? 256 : 512));
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem) + warp * RR_P2;
  const int g = lane % RR_G, grp = lane / RR_G;
  for (int64_t row = blockIdx.x * (int64_t)RR_WARPS + warp; row < m;
       row += (int64_t)gridDim.x * RR_WARPS) {
    const int32_t* ids = sids + row * Lp;
    const uint4 q = g < NC ? __ldg(reinterpret_cast<const uint4*>(U + row * (DW * 4)) + g)
                           : make_uint4(0u, 0u, 0u, 0u);
    int cnt = 0;
    for (int t0 = 0; t0 < Lp; t0 += 32 / RR_G) {
      const int t = t0 + grp;
      const int32_t id = t < Lp ? ids[t] : -1;
      uint32_t s = 0;
      if (id >= 0 && g < NC) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(U + (int64_t)id * (DW * 4)) + g);
        uint32_t a = __vabsdiffu4(q.x, v.x);
        s = __dp4a(a, a, s);
        a = __vabsdiffu4(q.y, v.y);
        s = __dp4a(a, a, s);
        a = __vabsdiffu4(q.z, v.z);
        s = __dp4a(a, a, s);
        a = __vabsdiffu4(q.w, v.w);
        s = __dp4a(a, a, s);
      }
#pragma unroll
      for (int o = 1; o < RR_G; o <<= 1) s += __shfl_xor_sync(FULL, s, o);
      if (g == 0 && t < Lp) keys[t] = id >= 0 ? pack_key((float)s, id) : ~0ull;
      cnt += __popc(__ballot_sync(FULL, g == 0 && t < Lp && id >= 0));
    }
    if (!rerank_sort_certify(keys, P2, cnt, row, Lp, L, sthr, sm, band, 1, fail_rows, fail_bound,
                             ctr, lane))
      continue;
    rerank_write(keys, row, L, out_ids, out_dist, lane);
  }
}

cudaError_t launch_rerank(const void* xr, const void* xc, int dtype, int64_t m, int d, int dpad,
                          const int32_t* sids, const uint32_t* sthr, int Lp, int L,
                          const ScreenModel& sm, float band, int exact, int32_t* out_ids,
                          float* out_dist, int32_t* fail_rows, float* fail_bound, Counters* ctr,
                          const uint8_t* u8, int u8w, cudaStream_t s) {
  if (u8 && exact && xr == xc && Lp <= RR_P2) {  // 8-bit rows of the same points
    const size_t sh8 = RR_WARPS * RR_P2 * 8;
    const int grid8 = (int)std::min<int64_t>((m + RR_WARPS - 1) / RR_WARPS, (int64_t)num_sms() * 32);
#define CNG_RU(DW)                                                                                 \
    if (u8w == DW) {                                                                               \
      cudaFuncSetAttribute(rerank_u8_kernel<DW>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                           (int)sh8);                                                              \
      count_launch();                                                                              \
      rerank_u8_kernel<DW><<<grid8, RR_WARPS * 32, sh8, s>>>(u8, m, sids, sthr, Lp, L, sm, band,   \
                                                             out_ids, out_dist, fail_rows,         \
                                                             fail_bound, ctr);                     \
      return cudaGetLastError();                                                                   \
    }
    CNG_RU(8)
    CNG_RU(16)
    CNG_RU(24)
    CNG_RU(32)
#undef CNG_RU
  }
  // rows wider than 256 (FP32 storage, up to 1024): the query slice in registers (wide path)
  const int nq4 = dtype == CNG_F32 && dpad > 256 ? (dpad / 4 + 31) / 32 : 0;
  const int NQ = nq4 == 0 ? 0 : (nq4 <= 4 ? 4 : (nq4 <= 8 ? 8 : 0));
  size_t sh = RR_WARPS * (RR_P2 * 8 + RR_RUN * 8 + 96 * 4) + (NQ ? 0 : RR_WARPS * dpad * sizeof(float));
  int grid = (int)std::min<int64_t>((m + RR_WARPS - 1) / RR_WARPS, (int64_t)num_sms() * 32);
#define CNG_RR(T, Q)                                                                          \
  do {                                                                                        \
    cudaFuncSetAttribute(rerank_kernel<T, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh); \
    count_launch();                                                                           \
    rerank_kernel<T, Q><<<grid, RR_WARPS * 32, sh, s>>>((const T*)xr, (const T*)xc, m, d, dpad, sids, \
                                                        sthr, Lp, L, sm, band, exact, out_ids, \
                                                        out_dist, fail_rows, fail_bound, ctr); \
  } while (0)
  if (dtype == CNG_F32) {
    if (NQ == 8)
      CNG_RR(float, 8);
    else if (NQ == 4)
      CNG_RR(float, 4);
    else
      CNG_RR(float, 0);
  } else {
    CNG_RR(__half, 0);
  }
#undef CNG_RR
  return cudaGetLastError();
}

// ============================================================================================
// rescan: exact candidate list for rows the certification rejected
// ============================================================================================
// One CTA per listed row.  `bound` is an upper bound on the row's true L-th smallest squared
// distance (K2 stores its L-th FP32 candidate value times (1 + error bound)).  Every column
// whose FP32 squared distance is <= bound * (1 + eps) is collected -- a superset of the true
// top-L -- and the collected set is ordered by the canonical (FP64 squared distance, id).  If
// more than RS_CAP columns qualify, the bound is lowered to the L-th smallest collected
// value (still an upper bound: L real points lie at or below it) and the scan repeats.
constexpr int RS_CAP = 4096;

CNG_DEV bool dk_less(double a, int32_t ia, double b, int32_t ib) {
  return a < b || (a == b && ia < ib);
}

CNG_DEV void cta_bitonic_dk(double* v, int32_t* id, int P2) {
  for (int k = 2; k <= P2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = (i & k) == 0;
          bool gt = dk_less(v[ixj], id[ixj], v[i], id[i]);
          if (gt == up) {
            double tv = v[i]; v[i] = v[ixj]; v[ixj] = tv;
            int32_t ti = id[i]; id[i] = id[ixj]; id[ixj] = ti;
          }
        }
      }
      __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
rescan_kernel(const T* __restrict__ Xr, const T* __restrict__ Xc, int64_t m, int64_t n, int d,
              int dpad, int self_excl, int L, const int32_t* __restrict__ fail_rows,
              const float* __restrict__ fail_bound, Counters* ctr, int32_t* __restrict__ out_ids,
              float* __restrict__ out_dist) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* v64 = reinterpret_cast<double*>(smem);               // RS_CAP
  int32_t* ids = reinterpret_cast<int32_t*>(v64 + RS_CAP);      // RS_CAP
  float* q = reinterpret_cast<float*>(ids + RS_CAP);            // dpad
  __shared__ int cnt;
  const int nf = ctr->nfail;
  const float eps = (float)(dpad + 8) * 5.9604645e-8f;
  for (int f = blockIdx.x; f < nf; f += gridDim.x) {
    const int64_t row = fail_rows[f];
    load_row(q, Xr + row * dpad, dpad, threadIdx.x, blockDim.x);
    float bound = fail_bound[f];
    int c = 0;
    for (int attempt = 0; attempt < 16; ++attempt) {
      if (threadIdx.x == 0) cnt = 0;
      __syncthreads();
      const float lim = bound * (1.f + 2.f * eps);
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        if (self_excl && j == row) continue;
        const T* y = Xc + j * dpad;
        float s = 0.f;
        for (int cc = 0; cc < dpad; ++cc) {
          float t = q[cc] - to_f(y[cc]);
          s = fmaf(t, t, s);
        }
        if (s <= lim) {
          int slot = atomicAdd(&cnt, 1);
          if (slot < RS_CAP) { v64[slot] = (double)s; ids[slot] = (int32_t)j; }
        }
      }
      __syncthreads();
      c = cnt;
      if (c <= RS_CAP) break;
      // too many: lower the bound to the L-th smallest FP32 value among those collected
      cta_bitonic_dk(v64, ids, RS_CAP);
      bound = (float)v64[L - 1] * (1.f + 2.f * eps);
      __syncthreads();
    }
    if (c > RS_CAP) {
      if (threadIdx.x == 0) set_status(&ctr->status, ST_CERT);
      c = RS_CAP;
    }
    int P2 = 1;
    while (P2 < c) P2 <<= 1;
    for (int t = threadIdx.x; t < P2; t += blockDim.x) {
      if (t < c) {
        v64[t] = canon_dist(Xr + row * dpad, Xc + (int64_t)ids[t] * dpad, d);
      } else {
        v64[t] = INFINITY;
        ids[t] = 0x7fffffff;
      }
    }
    __syncthreads();
    cta_bitonic_dk(v64, ids, P2);
    for (int t = threadIdx.x; t < L; t += blockDim.x) {
      out_ids[row * L + t] = t < c ? ids[t] : -1;
      out_dist[row * L + t] = t < c ? (float)v64[t] : INFINITY;
    }
    __syncthreads();
  }
}

cudaError_t launch_rescan(const void* xr, const void* xc, int dtype, int64_t m, int64_t n, int d,
                          int dpad, int self_excl, int L, const int32_t* fail_rows,
                          const float* fail_bound, Counters* ctr, int32_t* out_ids,
                          float* out_dist, cudaStream_t s) {
  size_t sh = RS_CAP * 8 + RS_CAP * 4 + dpad * 4;
  int grid = num_sms() * 2;
  if (dtype == CNG_F32) {
    cudaFuncSetAttribute(rescan_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch();
    rescan_kernel<float><<<grid, 256, sh, s>>>((const float*)xr, (const float*)xc, m, n, d, dpad,
                                               self_excl, L, fail_rows, fail_bound, ctr, out_ids,
                                               out_dist);
  } else {
    cudaFuncSetAttribute(rescan_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch();
    rescan_kernel<__half><<<grid, 256, sh, s>>>((const __half*)xr, (const __half*)xc, m, n, d,
                                                dpad, self_excl, L, fail_rows, fail_bound, ctr,
                                                out_ids, out_dist);
  }
  return cudaGetLastError();
}

}  // namespace cng
