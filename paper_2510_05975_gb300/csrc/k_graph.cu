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
#include "prune_rule.cuh"
#include "prune_tc.h"

namespace cng {

constexpr int PR_THREADS = 256;
constexpr int PR_G = 8;                       // lanes per pair distance
constexpr int PR_GROUPS = PR_THREADS / PR_G;  // 32 pair distances in flight per CTA
constexpr int PR_VMAX = 2048;                 // merged-list capacity
constexpr int PR_STAGE_BYTES = 96 * 1024;     // candidate vectors staged in shared memory
constexpr int PR_MERGE_STAGE_BYTES = 64 * 1024;


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

// ---- register-resident sweep ------------------------------------------------------------------
// Candidate i belongs to group i % PR_GROUPS, slot i / PR_GROUPS; each lane of the group keeps
// DL4 16-byte chunks of the vector (float4 index f4_index(g, q)) in registers for the whole
// sweep, so a pair distance reads nothing but the current S member's slice, which its owner
// publishes in shared memory.  Slots without a live candidate in the warp are skipped.
template <typename T>
CNG_DEV int f4_index(int g, int q) {
  // float rows: 16-byte chunks g, g + 8, ...; half rows: 16-byte half chunks g, g + 8, ...,
  // each giving two float4
  return sizeof(T) == 4 ? g + PR_G * q : 2 * (g + PR_G * (q >> 1)) + (q & 1);
}

template <typename T, int DL4>
CNG_DEV void load_slice(const T* __restrict__ row, int g, float4* x) {
  if (sizeof(T) == 4) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int q = 0; q < DL4; ++q) x[q] = __ldg(r4 + g + PR_G * q);
  } else {
    const uint4* r8 = reinterpret_cast<const uint4*>(row);
#pragma unroll
    for (int q = 0; q < DL4; q += 2) {
      const uint4 u = __ldg(r8 + g + PR_G * (q >> 1));
      x[q] = h8lo(u);
      x[q + 1] = h8hi(u);
    }
  }
}

// Alg. 2 over ids/dist [0, nv) (nv <= NSLOT * PR_GROUPS, dpad == 32 DL4); returns |S| (in S).
template <typename T, int NSLOT, int DL4>
CNG_DEV int prune_sweep_reg(const T* __restrict__ Xs, int d, int dpad, int64_t p,
                            const int32_t* ids, const float* dist, uint8_t* flags, int32_t* S,
                            float* vq, int nv, const RuleArgs& ra, unsigned long long& ties) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = tid % PR_G, grp = tid / PR_G;
  float4 xr[NSLOT][DL4];
#pragma unroll
  for (int k = 0; k < NSLOT; ++k) {
    const int i = k * PR_GROUPS + grp;
    if (i < nv) {
      load_slice<T, DL4>(Xs + (int64_t)ids[i] * dpad, g, xr[k]);
    } else {
#pragma unroll
      for (int q = 0; q < DL4; ++q) xr[k][q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  for (int i = tid; i < nv; i += PR_THREADS) flags[i] = 0;
  __syncthreads();
  float4* vq4 = reinterpret_cast<float4*>(vq);
  int ns = 0, cur = -1;
  for (;;) {
    // the next member of S: first candidate after cur not pruned yet (same in every warp)
    int nxt = nv;
    for (int b = cur + 1; b < nv; b += 32) {
      const int t = b + lane;
      const unsigned bal = __ballot_sync(FULL, t < nv && !flags[t]);
      if (bal) {
        nxt = b + __ffs(bal) - 1;
        break;
      }
    }
    if (nxt >= nv) break;
    const int32_t v = ids[nxt];
    if (tid == 0) S[ns] = v;
    ++ns;
    cur = nxt;
    if (ns >= ra.R) break;
    if (grp == nxt % PR_GROUPS) {
      const int slot = nxt / PR_GROUPS;
#pragma unroll
      for (int k = 0; k < NSLOT; ++k)
        if (k == slot)
#pragma unroll
          for (int q = 0; q < DL4; ++q) vq4[f4_index<T>(g, q)] = xr[k][q];
    }
    __syncthreads();
    float4 vr[DL4];
#pragma unroll
    for (int q = 0; q < DL4; ++q) vr[q] = vq4[f4_index<T>(g, q)];
#pragma unroll
    for (int k = 0; k < NSLOT; ++k) {
      const int w = k * PR_GROUPS + grp;
      const bool live = w > cur && w < nv && !flags[w];
      if (!__any_sync(FULL, live)) continue;
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int q = 0; q < DL4; ++q) {
        if (q & 1)
          acc4(xr[k][q], vr[q], s1);
        else
          acc4(xr[k][q], vr[q], s0);
      }
      const float s = group_reduce<PR_G>(s0 + s1);
      if (live && g == 0) {
        const float Dwv = sqrtf(s);
        const float lhs = dist[w];
        const float rhs = ra.alpha32 * Dwv + ra.t32;
        bool pr;
        if (near_tie(lhs, rhs, ra.band)) {
          const T* xw = Xs + (int64_t)ids[w] * dpad;
          const double Dpw = canon_dist(Xs + p * dpad, xw, d);
          const double Dwv64 = canon_dist(xw, Xs + (int64_t)v * dpad, d);
          pr = rule64(Dpw, Dwv64, ra.alpha64, ra.t64);
          ++ties;
        } else {
          pr = lhs > rhs;
        }
        if (pr) flags[w] = 1;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  return ns;
}

// ---- 8-bit integer sweep --------------------------------------------------------------------
// For integer data whose coordinates span at most 255 (and d * span^2 < 2^24), the rows are
// kept as bytes u = x - min(x).  D(w,v)^2 = |u_w|^2 + |u_v|^2 - 2 <u_w, u_v> is then computed
// exactly in 32-bit integers (dp4a), so the FP32 D = sqrtf(D^2) equals the one of the direct
// FP32 difference form bit for bit (that sum is exact too), and every rule decision is the same.
// One candidate per thread (nv <= blockDim.x), its row in DW registers.  One barrier per member
// of S: every warp publishes its live mask and the row of its first live candidate (buffers
// alternate between steps), so after the barrier all threads know the next member and its row.
template <int DW>
struct U8Slot {
  uint4 row[DW / 4];
  uint32_t nrm, pad[3];
};

template <typename T, int DW>
CNG_DEV int prune_sweep_u8(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int d, int dpad,
                           int64_t p, const int32_t* ids, const float* dist, int32_t* S,
                           U8Slot<DW>* slots /* [2][warps] */, unsigned* masks /* [2][warps] */,
                           int nv, const RuleArgs& ra, unsigned long long& ties) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  uint4 wv[DW / 4];
  uint32_t nrm = 0;
  const bool have = tid < nv;
  float mydist = 0.f;
  int32_t myid = 0;
  if (have) {
    myid = ids[tid];
    mydist = dist[tid];
    const uint4* r = reinterpret_cast<const uint4*>(U + (int64_t)myid * (DW * 4));
#pragma unroll
    for (int q = 0; q < DW / 4; ++q) {
      wv[q] = __ldg(r + q);
      nrm = __dp4a(wv[q].x, wv[q].x, nrm);
      nrm = __dp4a(wv[q].y, wv[q].y, nrm);
      nrm = __dp4a(wv[q].z, wv[q].z, nrm);
      nrm = __dp4a(wv[q].w, wv[q].w, nrm);
    }
  } else {
#pragma unroll
    for (int q = 0; q < DW / 4; ++q) wv[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  bool alive = have;
  int ns = 0, cur = -1, par = 0;
  for (;;) {
    const unsigned m = __ballot_sync(FULL, alive && tid > cur);
    if (m && lane == __ffs(m) - 1) {
      U8Slot<DW>& sl = slots[par * nwarps + warp];
#pragma unroll
      for (int q = 0; q < DW / 4; ++q) sl.row[q] = wv[q];
      sl.nrm = nrm;
    }
    if (lane == 0) masks[par * nwarps + warp] = m;
    __syncthreads();
    int nxt = -1;
    for (int w = 0; w < nwarps; ++w) {
      const unsigned mm = masks[par * nwarps + w];
      if (mm) {
        nxt = w * 32 + __ffs(mm) - 1;
        break;
      }
    }
    if (nxt < 0) break;
    const int32_t v = ids[nxt];
    if (tid == 0) S[ns] = v;
    ++ns;
    cur = nxt;
    if (ns >= ra.R) break;
    if (alive && tid > cur) {
      const U8Slot<DW>& sv = slots[par * nwarps + (nxt >> 5)];
      uint32_t dot = 0;
#pragma unroll
      for (int q = 0; q < DW / 4; ++q) {
        const uint4 y = sv.row[q];
        dot = __dp4a(wv[q].x, y.x, dot);
        dot = __dp4a(wv[q].y, y.y, dot);
        dot = __dp4a(wv[q].z, y.z, dot);
        dot = __dp4a(wv[q].w, y.w, dot);
      }
      const int32_t d2 = (int32_t)(nrm + sv.nrm) - 2 * (int32_t)dot;
      const float Dwv = sqrtf((float)d2);
      const float rhs = ra.alpha32 * Dwv + ra.t32;
      bool pr;
      if (near_tie(mydist, rhs, ra.band)) {
        const T* xw = Xs + (int64_t)myid * dpad;
        const double Dpw = canon_dist(Xs + p * dpad, xw, d);
        const double Dwv64 = canon_dist(xw, Xs + (int64_t)v * dpad, d);
        pr = rule64(Dpw, Dwv64, ra.alpha64, ra.t64);
        ++ties;
      } else {
        pr = mydist > rhs;
      }
      if (pr) alive = false;
    }
    par ^= 1;
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
  unsigned long long ties = 0, edges = 0, asteps = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    for (int i = threadIdx.x; i < L; i += PR_THREADS) {
      sm.ids[i] = cand[p * L + i];
      sm.dist[i] = cdist[p * L + i];
    }
    __syncthreads();
    if (nstage) stage_vectors(Xs, dpad, sm.ids, nstage, sm.stage);
    __syncthreads();
    int steps;
    int ns = prune_with_rule(
        ra, [&](const RuleArgs& r) { return prune_sweep(Xs, d, dpad, p, sm, L, nstage, r, ties); },
        &steps);
    asteps += steps;
    for (int i = threadIdx.x; i < ra.R; i += PR_THREADS) fwd[p * ra.R + i] = i < ns ? sm.S[i] : -1;
    if (threadIdx.x == 0) fdeg[p] = ns;
    edges += ns;
    __syncthreads();
  }
  // per-thread tie counts (only group leaders count) -> one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if ((threadIdx.x & 31) == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (threadIdx.x == 0 && asteps) atomicAdd(&ctr->alpha_steps, asteps);
  (void)edges;
}

template <typename T, int NSLOT, int DL4>
__global__ void __launch_bounds__(PR_THREADS)
prune_fwd_reg_kernel(const T* __restrict__ Xs, int64_t n, int d, int dpad,
                     const int32_t* __restrict__ cand, const float* __restrict__ cdist, int L,
                     RuleArgs ra, int32_t* __restrict__ fwd, int32_t* __restrict__ fdeg,
                     Counters* ctr) {
  __shared__ int32_t s_ids[NSLOT * PR_GROUPS];
  __shared__ float s_dist[NSLOT * PR_GROUPS];
  __shared__ uint8_t s_flags[NSLOT * PR_GROUPS];
  __shared__ int32_t s_S[64];
  __shared__ __align__(16) float s_vq[DL4 * 32 * 4];
  unsigned long long ties = 0, asteps = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    for (int i = threadIdx.x; i < L; i += PR_THREADS) {
      s_ids[i] = cand[p * L + i];
      s_dist[i] = cdist[p * L + i];
    }
    __syncthreads();
    int steps;
    const int ns = prune_with_rule(ra, [&](const RuleArgs& r) {
      return prune_sweep_reg<T, NSLOT, DL4>(Xs, d, dpad, p, s_ids, s_dist, s_flags, s_S, s_vq, L, r,
                                            ties);
    }, &steps);
    asteps += steps;
    for (int i = threadIdx.x; i < ra.R; i += PR_THREADS) fwd[p * ra.R + i] = i < ns ? s_S[i] : -1;
    if (threadIdx.x == 0) fdeg[p] = ns;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if ((threadIdx.x & 31) == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (threadIdx.x == 0 && asteps) atomicAdd(&ctr->alpha_steps, asteps);
}

template <typename T, int DW>
__global__ void __launch_bounds__(256)
prune_fwd_u8_kernel(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int64_t n, int d,
                    int dpad, const int32_t* __restrict__ cand, const float* __restrict__ cdist,
                    int L, RuleArgs ra, int32_t* __restrict__ fwd, int32_t* __restrict__ fdeg,
                    Counters* ctr) {
  __shared__ int32_t s_ids[256];
  __shared__ float s_dist[256];
  __shared__ int32_t s_S[64];
  __shared__ U8Slot<DW> s_slots[2 * 8];
  __shared__ unsigned s_masks[2 * 8];
  unsigned long long ties = 0, asteps = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      s_ids[i] = cand[p * L + i];
      s_dist[i] = cdist[p * L + i];
    }
    __syncthreads();
    int steps;
    const int ns = prune_with_rule(ra, [&](const RuleArgs& r) {
      return prune_sweep_u8<T, DW>(U, Xs, d, dpad, p, s_ids, s_dist, s_S, s_slots, s_masks, L, r,
                                   ties);
    }, &steps);
    asteps += steps;
    for (int i = threadIdx.x; i < ra.R; i += blockDim.x) fwd[p * ra.R + i] = i < ns ? s_S[i] : -1;
    if (threadIdx.x == 0) fdeg[p] = ns;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if ((threadIdx.x & 31) == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (threadIdx.x == 0 && asteps) atomicAdd(&ctr->alpha_steps, asteps);
}

template <typename T>
static bool launch_prune_u8(const uint8_t* U, int dw, const T* xs, int64_t n, int d, int dpad,
                            const int32_t* cand, const float* cdist, int L, const RuleArgs& ra,
                            int32_t* fwd, int32_t* fdeg, Counters* ctr, cudaStream_t s) {
  if (!U || L > 256) return false;
  const int threads = (L + 31) / 32 * 32;
  const int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * (2048 / threads));
#define CNG_PU(DW)                                                                                 \
  if (dw == DW) {                                                                                  \
    count_launch();                                                                                \
    prune_fwd_u8_kernel<T, DW><<<grid, threads, 0, s>>>(U, xs, n, d, dpad, cand, cdist, L, ra, fwd, \
                                                        fdeg, ctr);                                \
    return true;                                                                                   \
  }
  CNG_PU(8)
  CNG_PU(16)
  CNG_PU(24)
  CNG_PU(32)
#undef CNG_PU
  return false;
}

// Register-resident variants: (slots, 16-byte chunks per lane) with slots * chunks <= 18.
template <typename T>
static bool launch_prune_reg(const T* xs, int64_t n, int d, int dpad, const int32_t* cand,
                             const float* cdist, int L, const RuleArgs& ra, int32_t* fwd,
                             int32_t* fdeg, Counters* ctr, cudaStream_t s) {
  const int dl4 = dpad / 32, ns = (L + PR_GROUPS - 1) / PR_GROUPS;
  const int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 16);
#define CNG_PR(NS, DL)                                                                          \
  if (dl4 == DL && ns <= NS) {                                                                  \
    count_launch();                                                                             \
    prune_fwd_reg_kernel<T, NS, DL><<<grid, PR_THREADS, 0, s>>>(xs, n, d, dpad, cand, cdist, L, \
                                                                ra, fwd, fdeg, ctr);            \
    return true;                                                                                \
  }
  if constexpr (sizeof(T) == 4) {
    if (dpad % 32 == 0) {
      CNG_PR(4, 4)
      CNG_PR(4, 3)
      CNG_PR(6, 3)
      CNG_PR(4, 2)
      CNG_PR(8, 2)
      CNG_PR(4, 1)
      CNG_PR(8, 1)
    }
  } else {
    if (dpad % 64 == 0) {
      CNG_PR(4, 4)
      CNG_PR(4, 2)
      CNG_PR(8, 2)
    }
  }
#undef CNG_PR
  return false;
}

cudaError_t launch_prune_fwd(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* cand, const float* cdist, int L, double alpha,
                             double tau, const AlphaGrid& ag, int R, float band, int32_t* fwd, int32_t* fdeg,
                             Counters* ctr, const uint8_t* u8, int u8_words, float* half_norms,
                             cudaStream_t s) {
  RuleArgs ra = rule_args(alpha, tau, R, band, R, ag);
  if (gram_prune_ok(u8, u8_words, L, R))  // 8-bit rows, lists of <= 128: Gram tile on tcgen05
    return launch_prune_gram_u8(u8, u8_words, xs, dtype, n, d, dpad, cand, cdist, L, ra, fwd, fdeg,
                                ctr, s);
  if (half_norms && gram_prune_f16_ok(dtype, dpad, L, R, ag.imax >= 0))  // FP16 rows, same tile
    return launch_prune_gram_f16(xs, n, d, dpad, cand, cdist, L, ra, fwd, fdeg, half_norms, ctr, s);
  if (!u8 && pairs_prune_ok(L, R, ag.imax >= 0))  // float rows: all pairs on CUDA cores
    return launch_prune_pairs(xs, dtype, n, d, dpad, cand, cdist, L, ra, fwd, fdeg, ctr, s);
  if (dtype == CNG_F32 ? launch_prune_u8(u8, u8_words, (const float*)xs, n, d, dpad, cand, cdist, L,
                                         ra, fwd, fdeg, ctr, s)
                       : launch_prune_u8(u8, u8_words, (const __half*)xs, n, d, dpad, cand, cdist,
                                         L, ra, fwd, fdeg, ctr, s))
    return cudaGetLastError();
  if (dtype == CNG_F32 ? launch_prune_reg((const float*)xs, n, d, dpad, cand, cdist, L, ra, fwd,
                                          fdeg, ctr, s)
                       : launch_prune_reg((const __half*)xs, n, d, dpad, cand, cdist, L, ra, fwd,
                                          fdeg, ctr, s))
    return cudaGetLastError();
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

// ---- 8-bit rows for integer data ----------------------------------------------------------------
// U[i][c] = x[i][c] - vmin (c < d), 0 in the padding up to 4 dw bytes; requires integer values
// in [vmin, vmin + 255].
template <typename T>
__global__ void to_u8_kernel(const T* __restrict__ xs, int64_t n, int d, int dpad, float vmin,
                             int dw, uint8_t* __restrict__ U) {
  const int64_t total = n * (int64_t)(dw * 4);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (dw * 4);
    const int c = (int)(e - i * (dw * 4));
    U[e] = c < d ? (uint8_t)(int)(to_f(xs[i * dpad + c]) - vmin) : (uint8_t)0;
  }
}

int u8_words(int d) {
  const int w = (d + 15) / 16 * 4;
  return (w == 8 || w == 16 || w == 24 || w == 32) ? w : 0;
}

cudaError_t launch_to_u8(const void* xs, int dtype, int64_t n, int d, int dpad, float vmin, int dw,
                         uint8_t* U, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((n * dw * 4 + 255) / 256, (int64_t)num_sms() * 16);
  count_launch();
  if (dtype == CNG_F32)
    to_u8_kernel<float><<<grid, 256, 0, s>>>((const float*)xs, n, d, dpad, vmin, dw, U);
  else
    to_u8_kernel<__half><<<grid, 256, 0, s>>>((const __half*)xs, n, d, dpad, vmin, dw, U);
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
constexpr int PR_PREFIX = 512;  // entries of a large merged set ordered and pruned first

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
template <typename T, int NS, int DL>
CNG_DEV int merge_node(const T* __restrict__ Xs, int d, int dpad, int64_t p,
                       const int32_t* __restrict__ fwd, int nf, const int32_t* __restrict__ inl,
                       int64_t i0, int nin, const RuleArgs& ra, int exact, const MergeArrays& ar,
                       PruneSmem& sm, double* d64, int32_t* rid, int stage_cap, int* s_nv,
                       int32_t* __restrict__ adj_row, Counters* ctr, unsigned long long& ties,
                       unsigned long long& ordties, unsigned long long& repruned,
                       const MergeScratch& ms, int lim0) {
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
  // FP64 re-decision of near-tied neighbours in the order (warp 0), for the runs that start in
  // [from, lim); runs longer than PR_RUN (large merged sets of hubs with concentrated
  // distances) are recorded, up to 8 per pass, and re-sorted by the whole CTA, then warp 0
  // continues after the last recorded one.  Returns q >= lim: [0, q) is in (D, id) order and
  // keys[q - 1], keys[q] are not near-tied (or q = nv), so the entries beyond q all follow it.
  __shared__ int s_lr_start[8], s_lr_len[8], s_nlr, s_next, s_qend;
  auto resolve_runs = [&](int from, int lim) -> int {
    if (tid == 0) s_qend = lim;
    __syncthreads();
    while (!exact && from + 1 < nv && from < lim) {
      if (tid == 0) {
        s_nlr = 0;
        s_next = nv;
      }
      __syncthreads();
      if (warp == 0) {
        int i = from;
        while (i + 1 < nv && i < lim) {
          int s = -1;
          for (int b = i; b + 1 < nv && b < lim && s < 0; b += 32) {
            int t = b + lane;
            bool nt = t + 1 < nv && t < lim &&
                      near_tie(key_dist(ar.keys[t]), key_dist(ar.keys[t + 1]), ra.band);
            unsigned bal = __ballot_sync(FULL, nt);
            if (bal) s = b + __ffs(bal) - 1;
          }
          if (s < 0) break;
          int e = s + 1;
          while (e + 1 < nv && near_tie(key_dist(ar.keys[e]), key_dist(ar.keys[e + 1]), ra.band)) ++e;
          int len = e - s + 1;
          if (len > PR_RUN) {
            const bool full = s_nlr == 8;  // warp-uniform (written by lane 0 before a __syncwarp)
            if (full) {
              if (lane == 0) s_next = s;
              break;
            }
            __syncwarp();
            if (lane == 0) {
              s_lr_start[s_nlr] = s;
              s_lr_len[s_nlr] = len;
              ++s_nlr;
              s_qend = max(s_qend, e + 1);
            }
            __syncwarp();
            ++ordties;
            i = e + 1;
            continue;
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
            s_qend = max(s_qend, e + 1);
          }
          __syncwarp();
          ++ordties;
          i = e + 1;
        }
      }
      __syncthreads();
      // long runs: canonical distances of the whole run (in the id / dist arrays, free until
      // they are filled below), then an odd-even transposition sort of the run by (D, id)
      const int nlr = s_nlr;
      for (int r = 0; r < nlr; ++r) {
        const int s0 = s_lr_start[r], len = s_lr_len[r];
        double* D = reinterpret_cast<double*>(ar.ids);  // ids and dist: 8 bytes per entry, contiguous
        for (int t = tid; t < len; t += PR_THREADS)
          D[t] = canon_dist(Xs + p * dpad, Xs + (int64_t)key_id(ar.keys[s0 + t]) * dpad, d);
        __syncthreads();
        for (int ph = 0; ph < len; ++ph) {
          for (int t = 2 * tid + (ph & 1); t + 1 < len; t += 2 * PR_THREADS) {
            const uint64_t ka = ar.keys[s0 + t], kb = ar.keys[s0 + t + 1];
            if (D[t + 1] < D[t] || (D[t + 1] == D[t] && key_id(kb) < key_id(ka))) {
              const double tdv = D[t];
              D[t] = D[t + 1];
              D[t + 1] = tdv;
              ar.keys[s0 + t] = kb;
              ar.keys[s0 + t + 1] = ka;
            }
          }
          __syncthreads();
        }
      }
      from = s_next;
      __syncthreads();
    }
    __syncthreads();
    const int q = min(s_qend, nv);
    __syncthreads();
    return q;
  };
  // A set that will be pruned needs its order only as far as Alg. 2 reads it, which stops at R
  // kept entries: large sets are ordered and pruned on a prefix first, and only if the sweep
  // runs out of it with fewer than R kept is the whole set ordered and pruned again.  (With
  // Alg. 4's alpha steps an early step's count decides whether later steps run, so a sweep that
  // ran out of the prefix in any step would not do; those sets are ordered whole.)
  const bool prefix_first =
      nv > lim0 && nv > ra.R && ra.imax < 0 && !(ms.mlist && nv <= ms.stride);
  int from = 0, lim = prefix_first ? lim0 : nv, na = 0;
  for (;;) {
    const int q = resolve_runs(from, lim);
    for (int i = tid; i < nv; i += PR_THREADS) {
      ar.ids[i] = key_id(ar.keys[i]);
      ar.dist[i] = sqrtf(key_dist(ar.keys[i]));
    }
    __syncthreads();
    if (ms.mlist && nv > ra.R && nv <= ms.stride) {
      // listed in (D, id) order for the all-pairs re-prune, which writes the row and its degree
      for (int i = tid; i < nv; i += PR_THREADS) {
        ms.mlist[p * ms.stride + i] = ar.ids[i];
        ms.mdist[p * ms.stride + i] = ar.dist[i];
      }
      if (tid == 0) {
        ms.mlen[p] = nv;
        ms.rlist[atomicAdd(&ctr->nre, 1)] = (int32_t)p;
      }
      __syncthreads();
      return -1;
    }
    if (nv <= ra.R) {
      na = nv;
      for (int i = tid; i < nv; i += PR_THREADS) sm.S[i] = ar.ids[i];
      __syncthreads();
      break;
    }
    int steps;
    if (NS > 0 && q <= NS * PR_GROUPS) {
      na = prune_with_rule(ra, [&](const RuleArgs& r) {
        return prune_sweep_reg<T, (NS > 0 ? NS : 1), (DL > 0 ? DL : 1)>(
            Xs, d, dpad, p, ar.ids, ar.dist, ar.flags, sm.S, sm.vq, q, r, ties);
      }, &steps);
    } else {
      const int nstage = min(q, stage_cap);
      stage_vectors(Xs, dpad, ar.ids, nstage, sm.stage);
      __syncthreads();
      na = prune_with_rule(
          ra, [&](const RuleArgs& r) { return prune_sweep(Xs, d, dpad, p, sm, q, nstage, r, ties); },
          &steps);
    }
    if (na >= ra.R || q >= nv) {
      ++repruned;
      break;
    }
    from = q;  // the prefix ran out with fewer than R kept: order the rest, prune the whole set
    lim = nv;
  }
  for (int i = tid; i < ra.rs; i += PR_THREADS) adj_row[i] = i < na ? sm.S[i] : -1;
  __syncthreads();
  return na;
}

// Shared layout: vq, pq [dpad] | S [64] | d64 [PR_RUN] | rid [PR_RUN] | arrays | stage
template <typename T, bool BIG, int NS, int DL>
__global__ void __launch_bounds__(PR_THREADS)
merge_kernel(const T* __restrict__ Xs, int64_t n, int d, int dpad, const int32_t* __restrict__ fwd,
             const int32_t* __restrict__ fdeg, const int64_t* __restrict__ off,
             const int32_t* __restrict__ inl, RuleArgs ra, int exact, int32_t* __restrict__ adj,
             int32_t* __restrict__ deg, Counters* ctr, int32_t* __restrict__ big_list,
             unsigned char* __restrict__ big_scratch, int big_cap, MergeScratch ms) {
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
    int na = merge_node<T, NS, DL>(Xs, d, dpad, p, fwd + p * ra.R, nf, inl, i0, nin, ra, exact, ar, sm, d64,
                        rid, stage_cap, &s_nv, adj + p * ra.rs, ctr, ties, ordties, repruned, ms,
                        PR_PREFIX);
    if (na < 0) continue;  // listed for the all-pairs re-prune
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

// Phase 3 from 8-bit integer rows: merged sets of up to CAP entries per CTA of CAP threads, one
// entry per thread -- exact integer D(p,.)^2, (D, id) order by ranks, then the 8-bit sweep.
// Pass 1 (CAP 128) takes every node and defers larger sets to mid_list; pass 2 (CAP 256) takes
// mid_list and defers larger sets to big_list for the global-scratch pass.
template <typename T, int DW, int CAP>
__global__ void __launch_bounds__(CAP, 1024 / CAP)  // 64 registers: 32 warps per SM
merge_u8_kernel(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int64_t n, int d, int dpad,
                const int32_t* __restrict__ fwd, const int32_t* __restrict__ fdeg,
                const int64_t* __restrict__ off, const int32_t* __restrict__ inl, RuleArgs ra,
                int32_t* __restrict__ adj, int32_t* __restrict__ deg, Counters* ctr,
                int32_t* __restrict__ mid_list, int32_t* __restrict__ big_list) {
  constexpr bool SECOND = CAP > 128;
  __shared__ int32_t s_raw[CAP];
  __shared__ uint64_t s_key[CAP];
  __shared__ int32_t s_ids[CAP];
  __shared__ float s_dist[CAP];
  __shared__ int32_t s_S[64];
  __shared__ U8Slot<DW> s_slots[2 * (CAP / 32)];
  __shared__ uint4 s_p[DW / 4];
  __shared__ unsigned s_masks[2 * (CAP / 32)];
  __shared__ int s_nv;
  const int tid = threadIdx.x;
  unsigned long long ties = 0, repruned = 0, edges = 0, maxlist = 0;
  const int64_t count = SECOND ? (int64_t)ctr->nmid : n;
  for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
    const int64_t p = SECOND ? (int64_t)mid_list[q] : q;
    const int nf = fdeg[p];
    const int64_t i0 = off[p];
    const int nin = (int)(off[p + 1] - i0);
    if (nf + nin > CAP) {  // uniform: deferred to the next pass
      if (tid == 0) {
        if (SECOND)
          big_list[atomicAdd(&ctr->nbig, 1)] = (int32_t)p;
        else
          mid_list[atomicAdd(&ctr->nmid, 1)] = (int32_t)p;
      }
      continue;
    }
    maxlist = max(maxlist, (unsigned long long)(nf + nin));
    const int32_t* fp = fwd + p * ra.R;
    if (tid < nf) s_raw[tid] = fp[tid];
    if (tid == 0) s_nv = nf;
    if (tid < DW / 4) s_p[tid] = __ldg(reinterpret_cast<const uint4*>(U + p * (DW * 4)) + tid);
    __syncthreads();
    if (tid < nin) {  // in-neighbours not already in fwd(p)
      const int32_t u = inl[i0 + tid];
      bool dup = false;
      for (int j = 0; j < nf && !dup; ++j) dup = fp[j] == u;
      if (!dup) s_raw[atomicAdd(&s_nv, 1)] = u;
    }
    __syncthreads();
    const int nv = s_nv;
    // exact D(p, u)^2 and the (D, id) key of entry tid
    uint32_t d2 = 0;
    int32_t u = 0;
    if (tid < nv) {
      u = s_raw[tid];
      const uint4* r = reinterpret_cast<const uint4*>(U + (int64_t)u * (DW * 4));
      uint32_t nu = 0, np = 0, dot = 0;
#pragma unroll
      for (int q = 0; q < DW / 4; ++q) {
        const uint4 a = __ldg(r + q), b = s_p[q];
        nu = __dp4a(a.x, a.x, nu); nu = __dp4a(a.y, a.y, nu);
        nu = __dp4a(a.z, a.z, nu); nu = __dp4a(a.w, a.w, nu);
        np = __dp4a(b.x, b.x, np); np = __dp4a(b.y, b.y, np);
        np = __dp4a(b.z, b.z, np); np = __dp4a(b.w, b.w, np);
        dot = __dp4a(a.x, b.x, dot); dot = __dp4a(a.y, b.y, dot);
        dot = __dp4a(a.z, b.z, dot); dot = __dp4a(a.w, b.w, dot);
      }
      d2 = nu + np - 2u * dot;
      s_key[tid] = pack_key((float)d2, u);
    }
    __syncthreads();
    if (tid < nv) {  // rank among the distinct keys
      const uint64_t k = s_key[tid];
      int rank = 0;
      for (int j = 0; j < nv; ++j) rank += s_key[j] < k;
      s_ids[rank] = u;
      s_dist[rank] = sqrtf((float)d2);
    }
    __syncthreads();
    int na;
    if (nv <= ra.R) {
      na = nv;
      if (tid < nv) s_S[tid] = s_ids[tid];
      __syncthreads();
    } else {
      int steps;
      na = prune_with_rule(ra, [&](const RuleArgs& r) {
        return prune_sweep_u8<T, DW>(U, Xs, d, dpad, p, s_ids, s_dist, s_S, s_slots, s_masks, nv, r,
                                     ties);
      }, &steps);
      ++repruned;
    }
    int32_t* row = adj + p * ra.rs;
    for (int i = tid; i < ra.rs; i += blockDim.x) row[i] = i < na ? s_S[i] : -1;
    if (tid == 0) deg[p] = na;
    edges += na;
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if ((tid & 31) == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (tid == 0) {
    atomicAdd(&ctr->merge_repruned, repruned);
    atomicAdd(&ctr->edges, edges);
    atomicMax(&ctr->merge_max_list, maxlist);
  }
}

template <typename T, bool BIG, int NS, int DL>
static cudaError_t merge_t2(const void* xs, int64_t n, int d, int dpad, const int32_t* fwd,
                           const int32_t* fdeg, const int64_t* off, const int32_t* inl,
                           const RuleArgs& ra, int exact, int32_t* adj, int32_t* deg,
                           Counters* ctr, int32_t* big_list, unsigned char* big_scratch,
                           int big_cap, int grid, const MergeScratch& ms, cudaStream_t s) {
  const int stage_cap = PR_MERGE_STAGE_BYTES / (dpad * 4);
  size_t sh = 2 * (size_t)dpad * 4 + 256 + PR_RUN * 12 + (BIG ? 0 : (size_t)PR_VMAX * 17) +
              (size_t)stage_cap * dpad * 4 + 16;
  cudaFuncSetAttribute(merge_kernel<T, BIG, NS, DL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sh);
  count_launch();
  const MergeScratch mk = BIG ? MergeScratch{} : ms;
  merge_kernel<T, BIG, NS, DL><<<grid, PR_THREADS, sh, s>>>((const T*)xs, n, d, dpad, fwd, fdeg, off,
                                                            inl, ra, exact, adj, deg, ctr, big_list,
                                                            big_scratch, big_cap, mk);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mk.mlist)
    e = launch_merge_pairs(xs, sizeof(T) == 4 ? CNG_F32 : CNG_F16, n, d, dpad, mk, ra, adj, deg, ctr, s);
  return e;
}

// Merged lists of up to 128 entries are pruned from registers when 16-byte chunks per lane
// (dpad / 32) is 1..4 (even for half rows); longer lists and other widths use staged vectors.
template <typename T, bool BIG>
static cudaError_t merge_t(const uint8_t* U, int dw, const void* xs, int64_t n, int d, int dpad,
                           const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                           const int32_t* inl, const RuleArgs& ra, int exact, int32_t* adj,
                           int32_t* deg, Counters* ctr, int32_t* big_list,
                           unsigned char* big_scratch, int big_cap, int grid,
                           const MergeScratch& ms, cudaStream_t s) {
  const int dl4 = dpad % 32 == 0 ? dpad / 32 : 0;
  constexpr bool half = sizeof(T) == 2;
  if constexpr (!BIG) {
    if (U) {  // 8-bit integer rows: two passes (the second reads its node count on the device)
      const int g1 = (int)std::min<int64_t>(n, (int64_t)num_sms() * 16);
      const int g2 = num_sms() * 4;
      int32_t* mid_list = big_list + n;
      // first pass (sets of <= 128) on the tcgen05 Gram tile when the rule fits it
      const bool gram = gram_prune_ok(U, dw, 128, ra.R);
#define CNG_MU(DWV)                                                                                \
  if (dw == DWV) {                                                                                 \
    if (gram) {                                                                                    \
      cudaError_t e = launch_merge_gram_u8(U, dw, xs, sizeof(T) == 4 ? CNG_F32 : CNG_F16, n, d,    \
                                           dpad, fwd, fdeg, off, inl, ra, adj, deg, ctr, mid_list, \
                                           ms, s);                                                 \
      if (e != cudaSuccess) return e;                                                              \
    } else {                                                                                       \
      count_launch();                                                                              \
      merge_u8_kernel<T, DWV, 128><<<g1, 128, 0, s>>>(U, (const T*)xs, n, d, dpad, fwd, fdeg, off,  \
                                                      inl, ra, adj, deg, ctr, mid_list, big_list); \
    }                                                                                              \
    count_launch();                                                                                \
    merge_u8_kernel<T, DWV, 256><<<g2, 256, 0, s>>>(U, (const T*)xs, n, d, dpad, fwd, fdeg, off,    \
                                                    inl, ra, adj, deg, ctr, mid_list, big_list);   \
    return cudaGetLastError();                                                                     \
  }
      CNG_MU(8)
      CNG_MU(16)
      CNG_MU(24)
      CNG_MU(32)
#undef CNG_MU
    }
  }
#define CNG_MG(DLV)                                                                                \
  if constexpr (!half || DLV % 2 == 0) {                                                           \
    if (dl4 == DLV)                                                                                \
      return merge_t2<T, BIG, 4, DLV>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg,    \
                                      ctr, big_list, big_scratch, big_cap, grid, ms, s);           \
  }
  if constexpr (!BIG) {
    CNG_MG(1)
    CNG_MG(2)
    CNG_MG(3)
    CNG_MG(4)
  }
#undef CNG_MG
  return merge_t2<T, BIG, 0, 0>(xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj, deg, ctr,
                                big_list, big_scratch, big_cap, grid, ms, s);
}


cudaError_t launch_merge(const void* xs, int dtype, int64_t n, int d, int dpad,
                         const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                         const int32_t* inl, double alpha, double tau, const AlphaGrid& ag,
                         int R, float band, int exact, int32_t* adj, int32_t* deg, int rs,
                         Counters* ctr, int32_t* big_list, const uint8_t* u8, int u8_words,
                         const MergeScratch& ms, cudaStream_t s) {
  RuleArgs ra = rule_args(alpha, tau, R, band, rs, ag);
  int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 4);
  return dtype == CNG_F32
             ? merge_t<float, false>(u8, u8_words, xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact,
                                     adj, deg, ctr, big_list, nullptr, 0, grid, ms, s)
             : merge_t<__half, false>(u8, u8_words, xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact,
                                      adj, deg, ctr, big_list, nullptr, 0, grid, ms, s);
}

cudaError_t launch_merge_big(const void* xs, int dtype, int64_t n, int d, int dpad,
                             const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                             const int32_t* inl, double alpha, double tau, const AlphaGrid& ag,
                             int R, float band, int exact, int32_t* adj, int32_t* deg, int rs,
                             Counters* ctr, int32_t* big_list, int nbig, unsigned char* scratch,
                             int big_cap, int grid, cudaStream_t s) {
  RuleArgs ra = rule_args(alpha, tau, R, band, rs, ag);
  (void)nbig;
  return dtype == CNG_F32
             ? merge_t<float, true>(nullptr, 0, xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact, adj,
                                    deg, ctr, big_list, scratch, big_cap, grid, MergeScratch{}, s)
             : merge_t<__half, true>(nullptr, 0, xs, n, d, dpad, fwd, fdeg, off, inl, ra, exact,
                                     adj, deg, ctr, big_list, scratch, big_cap, grid, MergeScratch{},
                                     s);
}

}  // namespace cng
