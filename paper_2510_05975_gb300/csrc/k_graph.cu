// k_graph.cu -- pruning and reverse-edge merge of the alpha-CNG build (sm_103a).
//   K4 prune_fwd  Alg. 2 with the rule of Def. 2 (Eq. 1) on every exact candidate list,
//                 stopping at R kept points (Alg. 3 phase 2, fixed alpha)
//   K5 reverse    in-edge lists of the phase-2 graph (CSR: degree count, scan, scatter)
//   K6 merge      lazy pruning of Sec. 4.3: V'(p) = N+(p) U in(p); if |V'| > R prune V'
//                 once with the same rule, else keep V' in (D, id) order (Alg. 3 phase 3)
//
// Alg. 2 as sweeps: the kept set S grows in candidate order; when v joins S, every later
// candidate w that is still alive is tested against v alone (D(p,w) > alpha D(w,v) + t), in
// parallel across the CTA.  A candidate is thus tested against exactly the members of S that
// precede it until one prunes it -- the pairs Alg. 2 evaluates -- and the next member of S is
// the first candidate still alive.  Pair distances are computed only against members of S
// (the reuse observation of Sec. 4.3).  FP32 rule decisions inside the near-tie band are
// re-decided with the canonical FP64 distances.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"

namespace cng {

constexpr int PR_THREADS = 256;
constexpr int PR_G = 8;                       // lanes per pair distance
constexpr int PR_GROUPS = PR_THREADS / PR_G;  // 32 pair distances in flight per CTA
constexpr int PR_VMAX = 2048;                 // merged-list capacity
constexpr int PR_STAGE_BYTES = 96 * 1024;     // candidate vectors staged in shared memory
constexpr int PR_MERGE_STAGE_BYTES = 64 * 1024;

struct RuleArgs {
  float alpha32, t32, band;
  double alpha64, t64;
  int R;   // out-degree bound
  int rs;  // row stride of the final adjacency (R + connectivity slots)
};

CNG_DEV float part_sqdist_ss(const float* __restrict__ a, const float* __restrict__ b, int dpad,
                             int g) {
  float s0 = 0.f, s1 = 0.f;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  int nch = dpad >> 2, c = g;
  for (; c + PR_G < nch; c += 2 * PR_G) {
    acc4(a4[c], b4[c], s0);
    acc4(a4[c + PR_G], b4[c + PR_G], s1);
  }
  for (; c < nch; c += PR_G) acc4(a4[c], b4[c], s0);
  return s0 + s1;
}

// Shared-memory layout of one prune CTA.
struct PruneSmem {
  int32_t* ids;     // list ids in (D, id) order
  float* dist;      // FP32 D(p, .)
  uint8_t* flags;   // 1 = pruned
  int32_t* S;       // kept ids
  float* vq;        // current S member's vector (float)
  float* pq;        // p's vector (float)
  float* stage;     // staged list vectors (float), or nullptr
};

// Alg. 2 sweep over smem list [0, nv); returns |S| (S written to sm.S).
template <typename T>
CNG_DEV int prune_sweep(const T* __restrict__ Xs, int d, int dpad, int64_t p, const PruneSmem& sm,
                        int nv, int nstage, const RuleArgs& ra, unsigned long long& ties) {
  __shared__ int s_next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid % PR_G, grp = tid / PR_G;
  for (int i = tid; i < nv; i += PR_THREADS) sm.flags[i] = 0;
  __syncthreads();
  int ns = 0, cur = -1;
  for (;;) {
    if (warp == 0) {
      int nxt = nv;
      for (int b = cur + 1; b < nv; b += 32) {
        int t = b + lane;
        unsigned bal = __ballot_sync(FULL, t < nv && !sm.flags[t]);
        if (bal) { nxt = b + __ffs(bal) - 1; break; }
      }
      if (lane == 0) s_next = nxt;
    }
    __syncthreads();
    const int nxt = s_next;
    if (nxt >= nv) break;
    const int32_t v = sm.ids[nxt];
    if (tid == 0) sm.S[ns] = v;
    ++ns;
    cur = nxt;
    if (ns >= ra.R) break;
    // this S member's vector as floats
    if (cur < nstage) {
      for (int c = tid; c < dpad; c += PR_THREADS) sm.vq[c] = sm.stage[(size_t)cur * dpad + c];
    } else {
      load_row(sm.vq, Xs + (int64_t)v * dpad, dpad, tid, PR_THREADS);
    }
    __syncthreads();
    for (int w0 = cur + 1; w0 < nv; w0 += PR_GROUPS) {
      const int w = w0 + grp;
      const bool live = w < nv && !sm.flags[w];
      float s = 0.f;
      if (live) {
        s = w < nstage ? part_sqdist_ss(sm.vq, sm.stage + (size_t)w * dpad, dpad, g)
                       : part_sqdist<PR_G>(sm.vq, Xs + (int64_t)sm.ids[w] * dpad, dpad, g);
      }
      s = group_reduce<PR_G>(s);
      if (live && g == 0) {
        const float Dwv = sqrtf(s);
        const float lhs = sm.dist[w];
        const float rhs = ra.alpha32 * Dwv + ra.t32;
        bool pr;
        if (near_tie(lhs, rhs, ra.band)) {
          const T* xw = Xs + (int64_t)sm.ids[w] * dpad;
          double Dpw = canon_dist(Xs + p * dpad, xw, d);
          double Dwv64 = canon_dist(xw, Xs + (int64_t)v * dpad, d);
          pr = rule64(Dpw, Dwv64, ra.alpha64, ra.t64);
          ++ties;
        } else {
          pr = lhs > rhs;
        }
        if (pr) sm.flags[w] = 1;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  return ns;
}

template <typename T>
CNG_DEV void stage_vectors(const T* __restrict__ Xs, int dpad, const int32_t* ids, int nstage,
                           float* stage) {
  const int tid = threadIdx.x;
  if (sizeof(T) == 4) {
    const int cpr = dpad >> 2;
    for (int e = tid; e < nstage * cpr; e += PR_THREADS) {
      int i = e / cpr, c = e - i * cpr;
      reinterpret_cast<float4*>(stage + (size_t)i * dpad)[c] =
          __ldg(reinterpret_cast<const float4*>(Xs + (int64_t)ids[i] * dpad) + c);
    }
  } else {
    const int cpr = dpad >> 3;
    for (int e = tid; e < nstage * cpr; e += PR_THREADS) {
      int i = e / cpr, c = e - i * cpr;
      uint4 u = __ldg(reinterpret_cast<const uint4*>(Xs + (int64_t)ids[i] * dpad) + c);
      float4* d4 = reinterpret_cast<float4*>(stage + (size_t)i * dpad);
      d4[2 * c] = h8lo(u);
      d4[2 * c + 1] = h8hi(u);
    }
  }
}

// ---- K4 --------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(PR_THREADS)
prune_fwd_kernel(const T* __restrict__ Xs, int64_t n, int d, int dpad,
                 const int32_t* __restrict__ cand, const float* __restrict__ cdist, int L,
                 RuleArgs ra, int32_t* __restrict__ fwd, int32_t* __restrict__ fdeg, Counters* ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  PruneSmem sm;
  unsigned char* ptr = smem;
  sm.vq = reinterpret_cast<float*>(ptr); ptr += dpad * 4;
  sm.pq = nullptr;
  sm.ids = reinterpret_cast<int32_t*>(ptr); ptr += ((L * 4 + 15) / 16) * 16;
  sm.dist = reinterpret_cast<float*>(ptr); ptr += ((L * 4 + 15) / 16) * 16;
  sm.S = reinterpret_cast<int32_t*>(ptr); ptr += 64 * 4;
  sm.flags = reinterpret_cast<uint8_t*>(ptr); ptr += ((L + 15) / 16) * 16;
  const int nstage = (L * dpad * 4 <= PR_STAGE_BYTES) ? L : 0;
  sm.stage = nstage ? reinterpret_cast<float*>(ptr) : nullptr;
  unsigned long long ties = 0, edges = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    for (int i = threadIdx.x; i < L; i += PR_THREADS) {
      sm.ids[i] = cand[p * L + i];
      sm.dist[i] = cdist[p * L + i];
    }
    __syncthreads();
    if (nstage) stage_vectors(Xs, dpad, sm.ids, nstage, sm.stage);
    __syncthreads();
    int ns = prune_sweep(Xs, d, dpad, p, sm, L, nstage, ra, ties);
    for (int i = threadIdx.x; i < ra.R; i += PR_THREADS) fwd[p * ra.R + i] = i < ns ? sm.S[i] : -1;
    if (threadIdx.x == 0) fdeg[p] = ns;
    edges += ns;
    __syncthreads();
  }
  // per-thread tie counts (only group leaders count) -> one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if ((threadIdx.x & 31) == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  (void)edges;
}

cudaError_t launch_prune_fwd(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* cand, const float* cdist, int L, double alpha,
                             double tau, int R, float band, int32_t* fwd, int32_t* fdeg,
                             Counters* ctr, cudaStream_t s) {
  RuleArgs ra;
  ra.alpha64 = alpha;
  ra.t64 = (alpha + 1.0) * tau;
  ra.alpha32 = (float)alpha;
  ra.t32 = (float)ra.t64;
  ra.band = band;
  ra.R = R;
  ra.rs = R;
  size_t sh = dpad * 4 + 2 * (((size_t)L * 4 + 15) / 16) * 16 + 256 + ((L + 15) / 16) * 16;
  if ((size_t)L * dpad * 4 <= PR_STAGE_BYTES) sh += (size_t)L * dpad * 4;
  int per_sm = sh > 110 * 1024 ? 1 : 2;
  int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * per_sm * 4);
  if (dtype == CNG_F32) {
    cudaFuncSetAttribute(prune_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch();
    prune_fwd_kernel<float><<<grid, PR_THREADS, sh, s>>>((const float*)xs, n, d, dpad, cand, cdist,
                                                         L, ra, fwd, fdeg, ctr);
  } else {
    cudaFuncSetAttribute(prune_fwd_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch();
    prune_fwd_kernel<__half><<<grid, PR_THREADS, sh, s>>>((const __half*)xs, n, d, dpad, cand,
                                                          cdist, L, ra, fwd, fdeg, ctr);
  }
  return cudaGetLastError();
}

// ---- K5: reverse CSR -------------------------------------------------------------------------
__global__ void indeg_kernel(const int32_t* __restrict__ fwd, const int32_t* __restrict__ fdeg,
                             int64_t n, int R, int32_t* __restrict__ indeg) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  int64_t u = e / R;
  int j = (int)(e - u * R);
  if (j < fdeg[u]) atomicAdd(&indeg[fwd[e]], 1);
}

__global__ void max_indeg_kernel(const int32_t* __restrict__ indeg, int64_t n, Counters* ctr) {
  int mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, indeg[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&ctr->max_indeg, mx);
}

constexpr int SCAN_B = 1024;

// inclusive scan of one SCAN_B chunk per block -> off[i + 1]; block totals to blocksums
__global__ void scan_block_kernel(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ off,
                                  int64_t* __restrict__ blocksums) {
  __shared__ int64_t ws[32];
  int64_t i = blockIdx.x * (int64_t)SCAN_B + threadIdx.x;
  int64_t v = i < n ? in[i] : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) ws[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(FULL, w, o);
      if (lane >= o) w += t;
    }
    ws[lane] = w;
  }
  __syncthreads();
  if (warp > 0) v += ws[warp - 1];
  if (i < n) off[i + 1] = v;
  if (threadIdx.x == SCAN_B - 1) blocksums[blockIdx.x] = v;
}

__global__ void scan_sums_kernel(int64_t* blocksums, int64_t nb, int64_t* off) {
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int64_t b = 0; b < nb; ++b) {
      int64_t t = blocksums[b];
      blocksums[b] = acc;  // exclusive
      acc += t;
    }
    off[0] = 0;
  }
}

__global__ void scan_add_kernel(int64_t* __restrict__ off, int64_t n,
                                const int64_t* __restrict__ blocksums) {
  int64_t i = blockIdx.x * (int64_t)SCAN_B + threadIdx.x;
  if (i < n) off[i + 1] += blocksums[blockIdx.x];
}

__global__ void scatter_kernel(const int32_t* __restrict__ fwd, const int32_t* __restrict__ fdeg,
                               int64_t n, int R, const int64_t* __restrict__ off,
                               int32_t* __restrict__ cursor, int32_t* __restrict__ inl) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  int64_t u = e / R;
  int j = (int)(e - u * R);
  if (j < fdeg[u]) {
    int32_t v = fwd[e];
    int pos = atomicAdd(&cursor[v], 1);
    inl[off[v] + pos] = (int32_t)u;
  }
}

int64_t reverse_blocksums_len(int64_t n) { return (n + SCAN_B - 1) / SCAN_B; }

cudaError_t launch_reverse(const int32_t* fwd, const int32_t* fdeg, int64_t n, int R,
                           int32_t* indeg, int64_t* off, int32_t* cursor, int32_t* inl,
                           int64_t* blocksums, Counters* ctr, cudaStream_t s) {
  cudaMemsetAsync(indeg, 0, n * sizeof(int32_t), s);
  cudaMemsetAsync(cursor, 0, n * sizeof(int32_t), s);
  int64_t ne = n * R;
  int g = (int)((ne + 255) / 256);
  count_launch();
  indeg_kernel<<<g, 256, 0, s>>>(fwd, fdeg, n, R, indeg);
  count_launch();
  max_indeg_kernel<<<(int)std::min<int64_t>((n + 255) / 256, num_sms() * 4), 256, 0, s>>>(indeg, n, ctr);
  int64_t nb = reverse_blocksums_len(n);
  count_launch();
  scan_block_kernel<<<(int)nb, SCAN_B, 0, s>>>(indeg, n, off, blocksums);
  count_launch();
  scan_sums_kernel<<<1, 32, 0, s>>>(blocksums, nb, off);
  count_launch();
  scan_add_kernel<<<(int)nb, SCAN_B, 0, s>>>(off, n, blocksums);
  count_launch();
  scatter_kernel<<<g, 256, 0, s>>>(fwd, fdeg, n, R, off, cursor, inl);
  return cudaGetLastError();
}

// ---- K6: merge + lazy pruning ------------------------------------------------------------------
CNG_DEV void cta_bitonic64(uint64_t* a, int P2) {
  for (int k = 2; k <= P2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) { a[i] = y; a[ixj] = x; }
        }
      }
      __syncthreads();
    }
}

constexpr int PR_RUN = 256;  // longest near-tie run re-sorted in FP64

// Per-node working arrays of the merge (shared memory for ordinary nodes, global scratch for
// nodes whose merged set exceeds the shared capacity).
struct MergeArrays {
  uint64_t* keys;
  int32_t* ids;
  float* dist;
  uint8_t* flags;
  int cap;
};

// One node of phase 3: V'(p) = fwd(p) U in(p) without duplicates, sorted by (D(p,.), id) --
// FP32 keys, near-tied neighbours re-ordered by the canonical FP64 distance -- then kept as is
// if |V'| <= R, else pruned once with the rule (Sec. 4.3, lazy pruning).  Returns |adj(p)|.
template <typename T>
CNG_DEV int merge_node(const T* __restrict__ Xs, int d, int dpad, int64_t p,
                       const int32_t* __restrict__ fwd, int nf, const int32_t* __restrict__ inl,
                       int64_t i0, int nin, const RuleArgs& ra, int exact, const MergeArrays& ar,
                       PruneSmem& sm, double* d64, int32_t* rid, int stage_cap, int* s_nv,
                       int32_t* __restrict__ adj_row, Counters* ctr, unsigned long long& ties,
                       unsigned long long& ordties, unsigned long long& repruned) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid % PR_G, grp = tid / PR_G;
  sm.ids = ar.ids;
  sm.dist = ar.dist;
  sm.flags = ar.flags;
  if (tid == 0) *s_nv = nf;
  for (int i = tid; i < nf; i += PR_THREADS) ar.ids[i] = fwd[i];
  load_row(sm.pq, Xs + p * dpad, dpad, tid, PR_THREADS);
  __syncthreads();
  for (int i = tid; i < nin; i += PR_THREADS) {
    int32_t u = inl[i0 + i];
    bool dup = false;
    for (int j = 0; j < nf && !dup; ++j) dup = fwd[j] == u;
    if (!dup) {
      int slot = atomicAdd(s_nv, 1);
      if (slot < ar.cap) ar.ids[slot] = u;
    }
  }
  __syncthreads();
  int nv = *s_nv;
  if (nv > ar.cap) {
    if (tid == 0) set_status(&ctr->status, ST_OVF_MERGE);
    nv = ar.cap;
  }
  int P2 = 1;
  while (P2 < nv) P2 <<= 1;
  for (int i0g = 0; i0g < nv; i0g += PR_GROUPS) {
    int i = i0g + grp;
    float s = 0.f;
    if (i < nv) s = part_sqdist<PR_G>(sm.pq, Xs + (int64_t)ar.ids[i] * dpad, dpad, g);
    s = group_reduce<PR_G>(s);
    if (i < nv && g == 0) ar.keys[i] = pack_key(s, ar.ids[i]);
  }
  for (int i = nv + tid; i < P2; i += PR_THREADS) ar.keys[i] = ~0ull;
  __syncthreads();
  cta_bitonic64(ar.keys, P2);
  // FP64 re-decision of near-tied neighbours in the order (warp 0)
  if (!exact && warp == 0) {
    int i = 0;
    while (i + 1 < nv) {
      int s = -1;
      for (int b = i; b + 1 < nv && s < 0; b += 32) {
        int t = b + lane;
        bool nt = t + 1 < nv && near_tie(key_dist(ar.keys[t]), key_dist(ar.keys[t + 1]), ra.band);
        unsigned bal = __ballot_sync(FULL, nt);
        if (bal) s = b + __ffs(bal) - 1;
      }
      if (s < 0) break;
      int e = s + 1;
      while (e + 1 < nv && near_tie(key_dist(ar.keys[e]), key_dist(ar.keys[e + 1]), ra.band)) ++e;
      int len = e - s + 1;
      if (len > PR_RUN) {
        if (lane == 0) set_status(&ctr->status, ST_OVF_RUN);
        len = PR_RUN;
        e = s + len - 1;
      }
      for (int t = lane; t < len; t += 32) {
        rid[t] = key_id(ar.keys[s + t]);
        d64[t] = canon_dist(Xs + p * dpad, Xs + (int64_t)rid[t] * dpad, d);
      }
      __syncwarp();
      if (lane == 0) {  // insertion sort of the run by (D, id)
        for (int a = 1; a < len; ++a) {
          double dv = d64[a];
          int32_t iv = rid[a];
          uint64_t kv = ar.keys[s + a];
          int b = a - 1;
          while (b >= 0 && (d64[b] > dv || (d64[b] == dv && rid[b] > iv))) {
            d64[b + 1] = d64[b];
            rid[b + 1] = rid[b];
            ar.keys[s + b + 1] = ar.keys[s + b];
            --b;
          }
          d64[b + 1] = dv;
          rid[b + 1] = iv;
          ar.keys[s + b + 1] = kv;
        }
      }
      __syncwarp();
      ++ordties;
      i = e + 1;
    }
  }
  __syncthreads();
  for (int i = tid; i < nv; i += PR_THREADS) {
    ar.ids[i] = key_id(ar.keys[i]);
    ar.dist[i] = sqrtf(key_dist(ar.keys[i]));
  }
  __syncthreads();
  int na;
  if (nv <= ra.R) {
    na = nv;
    for (int i = tid; i < nv; i += PR_THREADS) sm.S[i] = ar.ids[i];
    __syncthreads();
  } else {
    const int nstage = min(nv, stage_cap);
    stage_vectors(Xs, dpad, ar.ids, nstage, sm.stage);
    __syncthreads();
    na = prune_sweep(Xs, d, dpad, p, sm, nv, nstage, ra, ties);
    ++repruned;
  }
  for (int i = tid; i < ra.rs; i += PR_THREADS) adj_row[i] = i < na ? sm.S[i] : -1;
  __syncthreads();
  return na;
}

// Shared layout: vq, pq [dpad] | S [64] | d64 [PR_RUN] | rid [PR_RUN] | arrays | stage
template <typename T, bool BIG>
__global__ void __launch_bounds__(PR_THREADS)
merge_kernel(const T* __restrict__ Xs, int64_t n, int d, int dpad, const int32_t* __restrict__ fwd,
             const int32_t* __restrict__ fdeg, const int64_t* __restrict__ off,
             const int32_t* __restrict__ inl, RuleArgs ra, int exact, int32_t* __restrict__ adj,
             int32_t* __restrict__ deg, Counters* ctr, int32_t* __restrict__ big_list,
             unsigned char* __restrict__ big_scratch, int big_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_nv;
  PruneSmem sm;
  unsigned char* ptr = smem;
  sm.vq = reinterpret_cast<float*>(ptr); ptr += dpad * 4;
  sm.pq = reinterpret_cast<float*>(ptr); ptr += dpad * 4;
  sm.S = reinterpret_cast<int32_t*>(ptr); ptr += 64 * 4;
  double* d64 = reinterpret_cast<double*>(ptr); ptr += PR_RUN * 8;
  int32_t* rid = reinterpret_cast<int32_t*>(ptr); ptr += PR_RUN * 4;
  MergeArrays ar;
  if (!BIG) {
    ar.cap = PR_VMAX;
    ar.keys = reinterpret_cast<uint64_t*>(ptr); ptr += PR_VMAX * 8;
    ar.ids = reinterpret_cast<int32_t*>(ptr); ptr += PR_VMAX * 4;
    ar.dist = reinterpret_cast<float*>(ptr); ptr += PR_VMAX * 4;
    ar.flags = reinterpret_cast<uint8_t*>(ptr); ptr += PR_VMAX;
  } else {
    unsigned char* g = big_scratch + (size_t)blockIdx.x * big_cap * 17;
    ar.cap = big_cap;
    ar.keys = reinterpret_cast<uint64_t*>(g);
    ar.ids = reinterpret_cast<int32_t*>(g + (size_t)big_cap * 8);
    ar.dist = reinterpret_cast<float*>(g + (size_t)big_cap * 12);
    ar.flags = g + (size_t)big_cap * 16;
  }
  const int stage_cap = PR_MERGE_STAGE_BYTES / (dpad * 4);
  sm.stage = reinterpret_cast<float*>(ptr);
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned long long ties = 0, ordties = 0, repruned = 0, edges = 0, maxlist = 0;
  const int64_t count = BIG ? (int64_t)ctr->nbig : n;
  for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int64_t p = BIG ? (int64_t)big_list[q] : q;
    const int nf = fdeg[p];
    const int64_t i0 = off[p];
    const int nin = (int)(off[p + 1] - i0);
    if (!BIG && nf + nin > PR_VMAX) {  // handled by the global-scratch pass
      if (tid == 0) big_list[atomicAdd(&ctr->nbig, 1)] = (int32_t)p;
      continue;
    }
    maxlist = max(maxlist, (unsigned long long)(nf + nin));
    int na = merge_node(Xs, d, dpad, p, fwd + p * ra.R, nf, inl, i0, nin, ra, exact, ar, sm, d64,
                        rid, stage_cap, &s_nv, adj + p * ra.rs, ctr, ties, ordties, repruned);
    if (tid == 0) deg[p] = na;
    edges += na;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if (lane == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (tid == 0) {
    if (ordties) atomicAdd(&ctr->order_ties, ordties);
    atomicAdd(&ctr->merge_repruned, repruned);
    atomicAdd(&ctr->edges, edges);
    atomicMax(&ctr->merge_max_list, maxlist);
  }
}

template <typename T, bool BIG>
static cudaError_t merge_t(const void* xs, int64_t n, int d, int dpad, const int32_t* fwd,
                           const int32_t* fdeg, const int64_t* off, const int32_t* inl,
                           const RuleArgs& ra, int exact, int32_t* adj, int32_t* deg,
                           Counters* ctr, int32_t* big_list, unsigned char* big_scratch,
                           int big_cap, int grid, cudaStream_t s) {
  const int stage_cap = PR_MERGE_STAGE_BYTES / (dpad * 4);
  size_t sh = 2 * (size_t)dpad * 4 + 256 + PR_RUN * 12 + (BIG ? 0 : (size_t)PR_VMAX * 17) +
              (size_t)stage_cap * dpad * 4 + 16;
  cudaFuncSetAttribute(merge_kernel<T, BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  count_launch();
  merge_kernel<T, BIG><<<grid, PR_THREADS, sh, s>>>((const T*)xs, n, d, dpad, fwd, fdeg, off, inl,
                                                    ra, exact, adj, deg, ctr, big_list,
                                                    big_scratch, big_cap);
  return cudaGetLastError();
}

static RuleArgs rule_args(double alpha, double tau, int R, float band, int rs) {
  RuleArgs ra;
  ra.rs = rs;
  ra.alpha64 = alpha;
  ra.t64 = (alpha + 1.0) * tau;
  ra.alpha32 = (float)alpha;
  ra.t32 = (float)ra.t64;
  ra.band = band;
  ra.R = R;
  return ra;
}

cudaError_t launch_merge(const void* xs, int dtype, int64_t n, int d, int dpad,
                         const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                         const int32_t* inl, double alpha, double tau, int R, float band,
                         int exact, int32_t* adj, int32_t* deg, int rs, Counters* ctr,
                         int32_t* big_list, cudaStream_t s) {
  RuleArgs ra = rule_args(alpha, tau, R, band, rs);
  int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 4);
  return dtype == CNG_F32
             ? merge_t<float, false>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg, ctr,
                                     big_list, nullptr, 0, grid, s)
             : merge_t<__half, false>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg,
                                      ctr, big_list, nullptr, 0, grid, s);
}

cudaError_t launch_merge_big(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                             const int32_t* inl, double alpha, double tau, int R, float band,
                             int exact, int32_t* adj, int32_t* deg, int rs, Counters* ctr,
                             int32_t* big_list, int nbig, unsigned char* scratch, int big_cap,
                             int grid, cudaStream_t s) {
  RuleArgs ra = rule_args(alpha, tau, R, band, rs);
  (void)nbig;
  return dtype == CNG_F32
             ? merge_t<float, true>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg, ctr,
                                    big_list, scratch, big_cap, grid, s)
             : merge_t<__half, true>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg, ctr,
                                     big_list, scratch, big_cap, grid, s);
}

}  // namespace cng
