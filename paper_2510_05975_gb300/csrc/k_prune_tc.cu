// k_prune_tc.cu -- Alg. 2 on whole-list pair tiles (sm_103a): the K4 prune of every candidate
// list (Alg. 3 phase 2b) and the lazy re-prune of the K6 merge (phase 3).
//   8-bit integer rows  tcgen05 Gram tile, exact (below); FP16 storage: the same tile from the
//                       stored rows, FP32-accumulated, with certified decision windows
//   other float rows    all pairs in 32 x 32 Gram blocks on CUDA cores, certified windows
//                       (pairs_prune_kernel, further down)
// All of them decide every pair of a list into bit masks and run Alg. 2 on the masks in one warp.
//
// Per point p its list V -- the L candidates in (D, id) order, or the merged set V'(p) ranked by
// (D, id) -- of up to 128 entries is staged as FP16 rows in 128-byte-swizzled shared memory, and
// tcgen05.mma (M = N = 128, K = the 8-bit row width, FP32 accumulators in 128 TMEM columns) forms
// the Gram matrix G = V V^T.  The rows hold u = x - min(x), integers in 0..255 with
// d * 255^2 < 2^24, so every product and every partial sum is an integer below 2^24 and the
// accumulators are exact: D(v_i, v_j)^2 = |u_i|^2 + |u_j|^2 - 2 G_ij is the same exact integer
// the SIMT sweep forms with dp4a.  The kernels check G_jj = |u_j|^2 on every entry and raise
// ST_SCREEN if the accumulation were ever inexact.
//
// Epilogue (4 warps; thread j reads TMEM lane j = entry j): every pair i < j is decided at once.
// Def. 2 / Eq. 1 -- v_i prunes v_j iff D(p,v_j) > alpha D(v_i,v_j) + t -- is taken in squared
// form, e = (D(p,v_j) - t)^2 - alpha^2 D(v_i,v_j)^2 in FP32 (one rounding after the exact
// integer D^2): e > w is a prune, |e| <= w a near-tie, with w = 2 band D(p,v_j) (D(p,v_j) - t)
// the squared image of the relative band (its FP32 error is below w / 12).  Entries with
// D(p,v_j) - t within 2 band D(p,v_j) of zero mark all their pairs near-tied.  The results are
// two 128-bit masks per entry ("pruned by", "near-tied with").
//
// Warp 0 then runs Alg. 2 on the masks: entry j joins S iff no member of S before it prunes it,
// until |S| = R.  Near-ties are re-decided with the canonical FP64 distances in the order Alg. 2
// meets them (the members of S before j, ascending, until one prunes j).
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "prune_rule.cuh"
#include "prune_tc.h"
#include "tc_ptx.cuh"

namespace cng {
namespace {

constexpr int GT_N = 128;                   // list entries per Gram tile (TMEM lanes and columns)
constexpr int GT_THREADS = 128;             // thread j <-> entry j <-> TMEM lane j
constexpr int GT_ABYTES = 2 * GT_N * 128;   // two 64-wide K atoms of 128 rows x 128 B (FP16)
constexpr uint32_t GT_IDESC = tcx::idesc_f16(GT_N, GT_N);
// Dynamic shared memory per CTA.  Also caps residency at 4 CTAs per SM, so the 4 x 128 TMEM
// columns the CTAs allocate always fit.
constexpr int GT_SMEM = 52 * 1024;

struct __align__(16) GramSmem {
  int32_t ids[GT_N];        // list in (D, id) order
  float dist[GT_N];         // FP32 D(p, v_j)
  float nrm[GT_N];          // |u_j|^2 (exact)
  uint32_t bp[GT_N][4];     // bit i of bp[j]: v_i prunes v_j (FP32-certain)
  uint32_t bt[GT_N][4];     // bit i of bt[j]: (v_i, v_j) near-tied
  int32_t S[64];
  // merge only
  uint64_t key[GT_N];
  int32_t raw[GT_N];
  uint4 prow[8];
  uint64_t bar;
  uint32_t tmem;
  int nv, ns, abort;
};
static_assert(GT_ABYTES + 1024 + sizeof(GramSmem) <= GT_SMEM, "Gram tile shared memory");

// One list's per-entry arrays in shared memory.
struct GramList {
  int32_t* ids;
  float* dist;
  float* nrm;
  uint32_t (*bp)[4];
  uint32_t (*bt)[4];
};
CNG_DEV GramList list_of(GramSmem& sm) { return GramList{sm.ids, sm.dist, sm.nrm, sm.bp, sm.bt}; }
static_assert(4 * (GT_SMEM + 1024) <= 228 * 1024 && 5 * (GT_SMEM + 1024) > 228 * 1024,
              "four CTAs per SM, never five");

// ---- rows -------------------------------------------------------------------------------------
template <int DW>
CNG_DEV void load_row(const uint8_t* __restrict__ U, int32_t id, uint4* w) {
  const uint4* src = reinterpret_cast<const uint4*>(U + (int64_t)id * (DW * 4));
#pragma unroll
  for (int g = 0; g < DW / 4; ++g) w[g] = __ldg(src + g);
}

template <int DW>
CNG_DEV uint32_t row_norm(const uint4* w) {
  uint32_t s = 0;
#pragma unroll
  for (int g = 0; g < DW / 4; ++g) {
    s = __dp4a(w[g].x, w[g].x, s);
    s = __dp4a(w[g].y, w[g].y, s);
    s = __dp4a(w[g].z, w[g].z, s);
    s = __dp4a(w[g].w, w[g].w, s);
  }
  return s;
}

template <int DW>
CNG_DEV uint32_t row_dot(const uint4* w, const uint4* q) {
  uint32_t s = 0;
#pragma unroll
  for (int g = 0; g < DW / 4; ++g) {
    const uint4 b = q[g];
    s = __dp4a(w[g].x, b.x, s);
    s = __dp4a(w[g].y, b.y, s);
    s = __dp4a(w[g].z, b.z, s);
    s = __dp4a(w[g].w, b.w, s);
  }
  return s;
}

// Two bytes of w (selected by sel) as an exact FP16 pair: 0x64bb is 1024 + b, minus 1024.
CNG_DEV uint32_t bytes_h2(uint32_t w, uint32_t sel) {
  uint32_t h = __byte_perm(w, 0x64646464u, sel);
  __half2 v = __hsub2(*reinterpret_cast<__half2*>(&h), __float2half2_rn(1024.f));
  return *reinterpret_cast<uint32_t*>(&v);
}

// Row r of the K-major operand: element k in atom k / 64, 16-byte chunk (k % 64) / 8 of the row's
// 128 bytes, chunk position XOR (r % 8) (the 128-byte swizzle).  One row per thread, so the
// eight rows of a quarter-warp hit eight different 16-byte bank groups.
template <int DW>
CNG_DEV void store_row_f16(const uint4* w, int r, unsigned char* A) {
#pragma unroll
  for (int g = 0; g < DW / 4; ++g) {
    const uint4 lo = make_uint4(bytes_h2(w[g].x, 0x4140), bytes_h2(w[g].x, 0x4342),
                                bytes_h2(w[g].y, 0x4140), bytes_h2(w[g].y, 0x4342));
    const uint4 hi = make_uint4(bytes_h2(w[g].z, 0x4140), bytes_h2(w[g].z, 0x4342),
                                bytes_h2(w[g].w, 0x4140), bytes_h2(w[g].w, 0x4342));
    const int s = (2 * g) & 7;
    unsigned char* row = A + (g >> 2) * (GT_N * 128) + r * 128;
    *reinterpret_cast<uint4*>(row + ((s ^ (r & 7)) << 4)) = lo;
    *reinterpret_cast<uint4*>(row + (((s + 1) ^ (r & 7)) << 4)) = hi;
  }
}

// G = V V^T: K in steps of 16 (32 bytes of an atom's row), A and B the same operand.
template <int DW>
CNG_DEV void issue_gram(const unsigned char* A, uint32_t tmem, uint64_t* bar) {
  tcx::fence_after();
  const uint32_t a0 = tcx::smem_u32(A);
#pragma unroll
  for (int k = 0; k < DW / 4; ++k) {
    const uint64_t a = tcx::desc_sw128(a0 + (k >> 2) * (GT_N * 128) + (k & 3) * 32);
    tcx::mma_f16(tmem, a, a, GT_IDESC, k > 0);
  }
  tcx::mma_commit(bar);
}

// ---- epilogue: masks ----------------------------------------------------------------------
// Thread j decides the pairs (i, j), i < j < V, from row j of G.  check: verify G_jj = |u_j|^2.
// With cE > 0 (FP16 rows: G from FP32 accumulation) D^2 carries an error of at most
// cE (|v_i|^2 + |v_j|^2); the window then adds alpha^2 times that and 2^-22 of the magnitudes, and
// the near-tie mask marks the pairs to decide again from the FP32 difference form (then FP64).
CNG_DEV void gram_masks(const GramList& sm, uint32_t tmem, int V, const RuleArgs& r, int warp, int lane,
                        uint32_t* check_status, float cE = 0.f) {
  const int j = warp * 32 + lane;
  const bool live = j < V;
  const float dj = live ? sm.dist[j] : 0.f;
  const float nj = live ? sm.nrm[j] : 0.f;
  const float tj = dj - r.t32;
  const float lim = 2.f * r.band * dj;
  const int cls = tj > lim ? 0 : (tj < -lim ? 1 : 2);  // squared test / never prunes / all near-tied
  const float T = tj * tj;
  const float w = 2.f * r.band * dj * tj;
  const float A2 = r.alpha32 * r.alpha32;
  const float A2cE = A2 * cE;
  const int nch = min(warp + 1, (V + 31) >> 5);  // warp-uniform; chunks past the row's own unused
  bool bad = false;
#pragma unroll 1
  for (int c = 0; c < nch; ++c) {
    const bool diag = c == warp;
    uint32_t pb = 0u, tb = 0u;
    float gjj = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // 16 columns per TMEM load (fewer live registers)
      float v[16];
      tcx::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32 + h * 16), v);
      const float* ni = sm.nrm + c * 32 + h * 16;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float g = v[k];
        const float d2 = (nj - g) + (ni[k] - g);  // exact for 8-bit rows: integers below 2^24
        const float e = fmaf(-A2, d2, T);
        float win = w;
        if (cE > 0.f) win = fmaf(2.384185791015625e-7f, fmaf(A2, fabsf(d2), T), fmaf(A2cE, nj + ni[k], w));
        pb |= e > win ? (1u << (h * 16 + k)) : 0u;
        tb |= fabsf(e) <= win ? (1u << (h * 16 + k)) : 0u;
      }
      if (diag) {
#pragma unroll
        for (int k = 0; k < 16; ++k) gjj = h * 16 + k == lane ? v[k] : gjj;
      }
    }
    const uint32_t valid = diag ? ((1u << lane) - 1u) : 0xffffffffu;
    if (live) {
      sm.bp[j][c] = cls == 0 ? (pb & valid) : 0u;
      sm.bt[j][c] = cls == 0 ? (tb & valid) : (cls == 2 ? valid : 0u);
    }
    if (check_status && diag && cE == 0.f) bad = live && gjj != nj;
  }
  if (bad) atomicOr(check_status, ST_SCREEN);
}

// ---- Alg. 2 on the masks (warp 0) -------------------------------------------------------------
template <typename T>
CNG_DEV bool prunes64(const GramList& sm, const T* __restrict__ Xs, int d, int dpad, int64_t p, int i,
                      int j, const RuleArgs& r) {
  const T* xj = Xs + (int64_t)sm.ids[j] * dpad;
  const double Dpj = canon_dist(Xs + p * dpad, xj, d);
  const double Dij = canon_dist(xj, Xs + (int64_t)sm.ids[i] * dpad, d);
  return rule64(Dpj, Dij, r.alpha64, r.t64);
}

// A pair the masks left open.  Exact D^2 (8-bit rows): a near-tie, re-decided in FP64.  FP16
// rows: D(v_i, v_j) from the FP32 difference form (4 accumulators, chain <= d / 4 + 3), then
// the rule with the relative band, FP64 inside it.  Counts the FP64 decisions.
template <typename T, bool EXACT>
CNG_DEV bool decide_pair(const GramList& sm, const T* __restrict__ Xs, int d, int dpad, int64_t p,
                         int i, int j, const RuleArgs& r, unsigned long long& ties) {
  if constexpr (!EXACT) {
    const T* xi = Xs + (int64_t)sm.ids[i] * dpad;
    const T* xj = Xs + (int64_t)sm.ids[j] * dpad;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int k = 0;
    for (; k + 4 <= d; k += 4) {
      float t;
      t = to_f(xi[k]) - to_f(xj[k]); s0 = fmaf(t, t, s0);
      t = to_f(xi[k + 1]) - to_f(xj[k + 1]); s1 = fmaf(t, t, s1);
      t = to_f(xi[k + 2]) - to_f(xj[k + 2]); s2 = fmaf(t, t, s2);
      t = to_f(xi[k + 3]) - to_f(xj[k + 3]); s3 = fmaf(t, t, s3);
    }
    for (; k < d; ++k) {
      const float t = to_f(xi[k]) - to_f(xj[k]);
      s0 = fmaf(t, t, s0);
    }
    const float Dij = sqrtf((s0 + s1) + (s2 + s3));
    const float rhs = r.alpha32 * Dij + r.t32;
    const float dj = sm.dist[j];
    if (!near_tie(dj, rhs, r.band)) return dj > rhs;
  }
  ++ties;
  return prunes64(sm, Xs, d, dpad, p, i, j, r);
}

CNG_DEV uint32_t word(const uint4& v, int q) { return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w; }

// Alg. 2 on the masks of the list [0, V), V <= 128 NV: bp[j] / bt[j] hold NV uint4 (4 NV words),
// word q covering the entries of chunk q (only q <= j / 32 are read).  Returns |S| (uniform over
// the warp); S written to S[].
template <typename T, bool EXACT, int NV>
CNG_DEV int mask_sweep(const GramList& gl, const uint4* bp, const uint4* bt, int32_t* S, int V,
                       const T* __restrict__ Xs, int d, int dpad, int64_t p, const RuleArgs& r, int lane,
                       unsigned long long& ties) {
  constexpr int NW = 4 * NV;
  const uint32_t* bpw = reinterpret_cast<const uint32_t*>(bp);
  const uint32_t* btw = reinterpret_cast<const uint32_t*>(bt);
  uint32_t K[NW];  // members of S by chunk (uniform)
#pragma unroll
  for (int q = 0; q < NW; ++q) K[q] = 0u;
  int ns = 0;
  const int nch = (V + 31) >> 5;
#pragma unroll 1
  for (int c = 0; c < nch; ++c) {
    const int j = c * 32 + lane;
    bool alive = j < V;
    // the entry's mask words: one list's four words held in registers, longer lists' read as used
    uint4 p4 = make_uint4(0u, 0u, 0u, 0u), t4 = p4;
    if (NV == 1 && alive) {
      p4 = bp[j];
      t4 = bt[j];
    }
    auto pw = [&](int q) { return NV == 1 ? word(p4, q) : bpw[j * NW + q]; };
    auto tw = [&](int q) { return NV == 1 ? word(t4, q) : btw[j * NW + q]; };
    if (alive && c > 0) {  // members of S from earlier chunks
      uint32_t hit = 0u, tie = 0u;
#pragma unroll
      for (int q = 0; q < NW; ++q)
        if (q < c) {
          hit |= pw(q) & K[q];
          tie |= tw(q) & K[q];
        }
      if (tie == 0u) {
        alive = hit == 0u;
      } else {  // ascending over the members that prune or tie, until one prunes
#pragma unroll
        for (int q = 0; q < NW; ++q) {
          if (q >= c || !alive) continue;
          const uint32_t bq = pw(q);
          uint32_t m = (bq | tw(q)) & K[q];
          while (m && alive) {
            const int b = __ffs(m) - 1;
            if ((bq >> b) & 1u) {
              alive = false;
            } else if (decide_pair<T, EXACT>(gl, Xs, d, dpad, p, q * 32 + b, j, r, ties)) {
              alive = false;
            }
            m &= m - 1u;
          }
        }
      }
    }
    // this chunk in order: the first alive entry joins S and tests the later ones
    const uint32_t bpc = j < V ? pw(c) : 0u, btc = j < V ? tw(c) : 0u;
    uint32_t kc = 0u;
    bool full = false;
    uint32_t live_m = __ballot_sync(FULL, alive);
    if (!__any_sync(FULL, alive && btc != 0u)) {
      // no near-tie inside the chunk: transpose the chunk's masks (prb[b] = the entries b prunes)
      // and run the greedy on bits, all lanes alike
      uint32_t prb[32];
#pragma unroll
      for (int b = 0; b < 32; ++b) prb[b] = __ballot_sync(FULL, (bpc >> b) & 1u);
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        if ((live_m >> b) & 1u) {
          kc |= 1u << b;
          live_m &= ~prb[b];
        }
      }
      const int room = r.R - ns;
      if (__popc(kc) >= room) {  // S fills up inside this chunk: its first `room` members
        uint32_t t = kc;
        for (int i = 1; i < room; ++i) t &= t - 1u;  // lowest set bit of t: the room-th member
        const int pos = __ffs(t) - 1;
        kc &= pos == 31 ? 0xffffffffu : ((2u << pos) - 1u);
        full = true;
      }
      if ((kc >> lane) & 1u) S[ns + __popc(kc & ((1u << lane) - 1u))] = gl.ids[c * 32 + lane];
      ns += __popc(kc);
      live_m = 0u;
    }
    while (live_m) {
      const int b = __ffs(live_m) - 1;
      kc |= 1u << b;
      if (lane == 0) S[ns] = gl.ids[c * 32 + b];
      ++ns;
      if (ns >= r.R) {
        full = true;
        break;
      }
      if (alive && lane > b) {
        if ((bpc >> b) & 1u) {
          alive = false;
        } else if ((btc >> b) & 1u) {
          if (decide_pair<T, EXACT>(gl, Xs, d, dpad, p, c * 32 + b, j, r, ties)) alive = false;
        }
      }
      live_m = __ballot_sync(FULL, alive) & ~((2u << b) - 1u);
    }
#pragma unroll
    for (int q = 0; q < NW; ++q)
      if (q == c) K[q] = kc;
    if (full) break;
  }
  __syncwarp();
  return ns;
}

// The Gram tiles' lists: 4 words per entry (V <= 128).
template <typename T, bool EXACT = true>
CNG_DEV int gram_sweep(const GramList& sm, int32_t* S, int V, const T* __restrict__ Xs, int d, int dpad,
                       int64_t p, const RuleArgs& r, int lane, unsigned long long& ties) {
  return mask_sweep<T, EXACT, 1>(sm, reinterpret_cast<const uint4*>(sm.bp),
                                 reinterpret_cast<const uint4*>(sm.bt), S, V, Xs, d, dpad, p, r, lane, ties);
}

// Masks and sweep for the list [0, V) with the fixed rule, or with Alg. 4's alpha steps.
// Returns |S| (uniform over the CTA); *steps = the last alpha step.
template <typename T>
CNG_DEV int gram_prune(GramSmem& sm, uint32_t tmem, int V, const T* __restrict__ Xs, int d, int dpad,
                       int64_t p, const RuleArgs& ra, int warp, int lane, uint32_t* status,
                       unsigned long long& ties, int* steps) {
  int ns = 0, i = 0;
  for (;; ++i) {
    const RuleArgs r = ra.imax >= 0 ? rule_step(ra, i) : ra;
    gram_masks(list_of(sm), tmem, V, r, warp, lane, i == 0 ? status : nullptr);
    __syncthreads();
    if (warp == 0) {
      const int k = gram_sweep(list_of(sm), sm.S, V, Xs, d, dpad, p, r, lane, ties);
      if (lane == 0) sm.ns = k;
    }
    __syncthreads();
    ns = sm.ns;
    if (ra.imax < 0 || 2 * ns >= ra.R || i >= ra.imax) break;
  }
  *steps = ra.imax >= 0 ? i : 0;
  return ns;
}

CNG_DEV unsigned char* align1024(unsigned char* p) {
  const uint32_t a = tcx::smem_u32(p);
  return p + (((a + 1023u) & ~1023u) - a);
}

CNG_DEV void gram_setup(GramSmem& sm, int warp) {
  if (threadIdx.x == 0) {
    tcx::mbar_init(&sm.bar, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tcx::tmem_alloc<GT_N>(&sm.tmem);
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
}

// Gram MMA of the staged rows and the wait for it; false (CTA-uniform) if the wait expired.
template <int DW>
CNG_DEV bool gram_mma(GramSmem& sm, const unsigned char* A, uint32_t tmem, uint32_t& phase,
                      uint32_t* status, int lane) {
  tcx::fence_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) issue_gram<DW>(A, tmem, &sm.bar);
  const bool ok = tcx::mbar_wait_warp(&sm.bar, phase);
  phase ^= 1u;
  if (!ok && lane == 0) {
    sm.abort = 1;
    atomicOr(status, ST_TIMEOUT);
  }
  tcx::fence_after();
  __syncthreads();
  return sm.abort == 0;
}

CNG_DEV void gram_teardown(GramSmem& sm, uint32_t tmem, uint32_t phase, int warp) {
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) {
    // after an expired wait, give the outstanding MMA one more bounded wait before freeing TMEM
    if (sm.abort) tcx::mbar_wait_warp(&sm.bar, phase ^ 1u);
    tcx::fence_after();
    tcx::tmem_dealloc<GT_N>(tmem);
  }
}

// ---- K4 ------------------------------------------------------------------------------------
template <typename T, int DW>
__global__ void __launch_bounds__(GT_THREADS)
prune_gram_u8_kernel(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int64_t n, int d,
                     int dpad, const int32_t* __restrict__ cand, const float* __restrict__ cdist,
                     int L, RuleArgs ra, int32_t* __restrict__ fwd, int32_t* __restrict__ fdeg,
                     Counters* ctr) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* A = align1024(smem_raw);
  GramSmem& sm = *reinterpret_cast<GramSmem*>(A + GT_ABYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  gram_setup(sm, warp);
  const uint32_t tmem = sm.tmem;
  uint32_t phase = 0;
  unsigned long long ties = 0, asteps = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    if (tid < L) {
      const int32_t id = cand[p * L + tid];
      sm.ids[tid] = id;
      sm.dist[tid] = cdist[p * L + tid];
      uint4 w[DW / 4];
      load_row<DW>(U, id, w);
      sm.nrm[tid] = (float)row_norm<DW>(w);
      store_row_f16<DW>(w, tid, A);
    }
    if (!gram_mma<DW>(sm, A, tmem, phase, &ctr->status, lane)) break;
    int steps;
    const int ns = gram_prune(sm, tmem, L, Xs, d, dpad, p, ra, warp, lane, &ctr->status, ties, &steps);
    asteps += steps;
    for (int t = tid; t < ra.R; t += GT_THREADS) fwd[p * ra.R + t] = t < ns ? sm.S[t] : -1;
    if (tid == 0) fdeg[p] = ns;
    tcx::fence_before();
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if (lane == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (tid == 0 && asteps) atomicAdd(&ctr->alpha_steps, asteps);
  gram_teardown(sm, tmem, phase, warp);
}

// ---- pipelined Gram prune (fixed alpha): K4, and the re-prune of K6 ---------------------------
// One job: rows q < count, each the list of point p = pts[q] (or q) -- list_stride entries of
// (D, id)-ordered ids and FP32 D(p, .) at row p, len[p] (or L) of them used -- pruned into
// out[p] (out_stride entries, -1 padded) and out_deg[p].
//
// Warps 0-3 (tile warps) read G(k) from TMEM into masks, stage row k+1's points into the operand
// tile and issue its Gram MMA; warp 4 (sweep warp) runs Alg. 2 on row k's masks and writes its
// list meanwhile.  Loads run ahead: row k+3's point, row k+2's list and row k+1's 8-bit rows are
// in flight while row k is decided.  Per-row arrays and masks are double-buffered; mbarriers
// order the roles:
//   mma       tcgen05.commit of the current Gram MMA           (tile warps wait)
//   ready[b]  masks of row k, b = k % 2, complete               (sweep warp waits)
//   freed[b]  the sweep of row k done: buffer b free again      (tile warps wait)
// Every wait is bounded; a warp whose wait expires records ST_TIMEOUT and skips its remaining
// work while still meeting every barrier, so the CTA always reaches its end.
struct GramJob {
  const int32_t* ids;
  const float* dist;
  int list_stride;
  const int32_t* len;  // per-point list length, or null: L
  int L;
  const int32_t* pts;  // row -> point, or null: the identity
  const int* count;    // number of rows (on the device), or null: n
  int64_t n;
  int32_t* out;
  int out_stride;
  int32_t* out_deg;
  int merge;           // count edges and re-pruned nodes (phase 3)
  const float* nrm;    // FP16 rows: |x|^2 of every point (FP32, one rounding)
};

constexpr int GP_THREADS = 160;

struct __align__(16) PipeSmem {
  int32_t ids[2][GT_N];
  float dist[2][GT_N];
  float nrm[2][GT_N];
  uint32_t bp[2][GT_N][4];
  uint32_t bt[2][GT_N][4];
  int32_t S[64];
  int64_t P[2];  // point of the row in each buffer
  int V[2];      // its list length
  uint64_t mma, ready[2], freed[2];
  uint32_t tmem;
  int abort;
};
static_assert(GT_ABYTES + 1024 + sizeof(PipeSmem) <= GT_SMEM, "pipelined Gram shared memory");

CNG_DEV GramList list_of(PipeSmem& sm, int b) {
  return GramList{sm.ids[b], sm.dist[b], sm.nrm[b], sm.bp[b], sm.bt[b]};
}

CNG_DEV void tile_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

CNG_DEV bool pipe_wait(PipeSmem& sm, uint64_t* bar, uint32_t parity, uint32_t* status, int lane) {
  if (tcx::mbar_wait_warp(bar, parity)) return true;
  if (lane == 0) {
    sm.abort = 1;
    atomicOr(status, ST_TIMEOUT);
  }
  __syncwarp();
  return false;
}

// Loads of one row ahead of its use: its point, its length and the thread's list entry.
struct RowAhead {
  int32_t p;
  int V;
  int32_t id;
  float dist;
  float nrm;  // FP16 rows: |x_id|^2
};

CNG_DEV int32_t job_point(const GramJob& J, int64_t q) { return J.pts ? J.pts[q] : (int32_t)q; }

CNG_DEV void job_list(const GramJob& J, RowAhead& r, int tid) {
  r.V = J.len ? J.len[r.p] : J.L;
  if (tid < J.list_stride) {  // (entries past V are read but unused)
    r.id = J.ids[(int64_t)r.p * J.list_stride + tid];
    r.dist = J.dist[(int64_t)r.p * J.list_stride + tid];
  }
}

// FP16 row r of the operand tile straight from global memory: K / 8 16-byte chunks, element k in
// atom k / 64, chunk (k % 64) / 8 of the row's 128 bytes, position XOR (r % 8).
template <int K>
CNG_DEV void stage_row_async(const __half* __restrict__ Xs, int dpad, int32_t id, int r,
                             unsigned char* A) {
  const uint4* src = reinterpret_cast<const uint4*>(Xs + (int64_t)id * dpad);
#pragma unroll
  for (int c = 0; c < K / 8; ++c)
    tcx::cp_async16(A + (c >> 3) * (GT_N * 128) + r * 128 + (((c & 7) ^ (r & 7)) << 4), src + c);
}

// The Gram error coefficient of K-element FP16 rows: |D^2_est - D^2| <= cE (|u|^2 + |v|^2) with
// products exact, at most K additions at 2^-22 of the magnitudes each in the accumulators, norms
// rounded once and three FP32 additions forming D^2.
constexpr float gram_ce(int K) { return (float)(4 * K + 8) * 5.9604644775390625e-8f; }

// HALF = false: 8-bit rows (U, K = 4 DW bytes per row, exact Gram values).  HALF = true: the
// FP16 point rows themselves (Xs, K = dpad <= 128), copied to the operand tile with cp.async,
// norms from J.nrm, decisions with the certified window of gram_ce(K).
template <typename T, int K, bool HALF>
__global__ void __launch_bounds__(GP_THREADS, 4)
gram_pipe_kernel(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int d, int dpad,
                 GramJob J, RuleArgs ra, Counters* ctr) {
  constexpr int DW = K / 4;
  static_assert(!HALF || K <= 128, "FP16 rows of at most two K atoms");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* A = align1024(smem_raw);
  PipeSmem& sm = *reinterpret_cast<PipeSmem*>(A + GT_ABYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tcx::mbar_init(&sm.mma, 1);
    for (int b = 0; b < 2; ++b) {
      tcx::mbar_init(&sm.ready[b], 1);
      tcx::mbar_init(&sm.freed[b], 1);
    }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tcx::tmem_alloc<GT_N>(&sm.tmem);
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = sm.tmem;
  const float cE = HALF ? gram_ce(K) : 0.f;
  // this CTA's rows q_k = blockIdx.x + k * gridDim.x, k < K
  const int64_t nq = J.count ? (int64_t)*J.count : J.n;
  const int64_t NK = (int64_t)blockIdx.x < nq ? (nq - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = gridDim.x;
  unsigned long long ties = 0, edges = 0;
  uint32_t issued = 0, completed = 0;  // Gram MMAs (meaningful in thread 0)
  if (warp < 4) {
    bool ok = true;
    RowAhead r1{0, 0, 0, 0.f, 0.f}, r2{0, 0, 0, 0.f, 0.f};  // rows k+1 and k+2
    int32_t p3 = 0;                                        // row k+3's point
    if (NK > 0) {  // row 0 staged, its MMA started; rows 1, 2 (lists) and 3 (point) in flight
      RowAhead r0{job_point(J, blockIdx.x), 0, 0, 0.f, 0.f};
      if (NK > 1) r1.p = job_point(J, blockIdx.x + G);
      if (NK > 2) r2.p = job_point(J, blockIdx.x + 2 * G);
      if (NK > 3) p3 = job_point(J, blockIdx.x + 3 * G);
      job_list(J, r0, tid);
      if (NK > 1) job_list(J, r1, tid);
      if (NK > 2) job_list(J, r2, tid);
      if (tid < r0.V) {
        sm.ids[0][tid] = r0.id;
        sm.dist[0][tid] = r0.dist;
        if constexpr (HALF) {
          sm.nrm[0][tid] = J.nrm[r0.id];
          stage_row_async<K>(reinterpret_cast<const __half*>(Xs), dpad, r0.id, tid, A);
        } else {
          uint4 w[DW / 4];
          load_row<DW>(U, r0.id, w);
          sm.nrm[0][tid] = (float)row_norm<DW>(w);
          store_row_f16<DW>(w, tid, A);
        }
      }
      if (tid == 0) {
        sm.P[0] = r0.p;
        sm.V[0] = r0.V;
      }
      if constexpr (HALF) tcx::cp_async_wait_all();
      tcx::fence_async_smem();
      tile_bar();
      if (tid == 0) {
        issue_gram<DW>(A, tmem, &sm.mma);
        ++issued;
      }
    }
    for (int64_t k = 0; k < NK; ++k) {
      const int b = (int)(k & 1);
      const bool next = k + 1 < NK;
      // loads ahead: rows of k+1 (8-bit rows), the list of k+3, the point of k+4
      uint4 w[HALF ? 1 : DW / 4];
      if constexpr (!HALF) {
        if (ok && next && tid < r1.V) load_row<DW>(U, r1.id, w);
      }
      float nrm1 = 0.f;
      if constexpr (HALF) {
        if (ok && next && tid < r1.V) nrm1 = J.nrm[r1.id];
      }
      RowAhead r3{p3, 0, 0, 0.f, 0.f};
      if (ok && k + 3 < NK) job_list(J, r3, tid);
      const int32_t p4 = (ok && k + 4 < NK) ? job_point(J, blockIdx.x + (k + 4) * G) : 0;
      if (ok) ok = pipe_wait(sm, &sm.mma, (uint32_t)(k & 1), &ctr->status, lane);
      if (ok && tid == 0) ++completed;
      tcx::fence_after();
      if constexpr (HALF) {  // the operand tile is free: row k+1's rows go in while G(k) is read
        if (ok && next && tid < r1.V)
          stage_row_async<K>(reinterpret_cast<const __half*>(Xs), dpad, r1.id, tid, A);
        tcx::cp_async_commit();
      }
      // masks of row k into buffer b, once row k-2's sweep released it
      if (ok && k >= 2) ok = pipe_wait(sm, &sm.freed[b], (uint32_t)(((k - 2) >> 1) & 1), &ctr->status, lane);
      if (ok) gram_masks(list_of(sm, b), tmem, sm.V[b], ra, warp, lane, &ctr->status, cE);
      tcx::fence_before();
      // row k+1 into buffer b ^ 1 (and the operand tile), once row k-1's sweep released it
      if (ok && next && k >= 1)
        ok = pipe_wait(sm, &sm.freed[b ^ 1], (uint32_t)(((k - 1) >> 1) & 1), &ctr->status, lane);
      if (ok && next) {
        if (tid < r1.V) {
          sm.ids[b ^ 1][tid] = r1.id;
          sm.dist[b ^ 1][tid] = r1.dist;
          if constexpr (HALF) {
            sm.nrm[b ^ 1][tid] = nrm1;
          } else {
            sm.nrm[b ^ 1][tid] = (float)row_norm<DW>(w);
            store_row_f16<DW>(w, tid, A);
          }
        }
        if (tid == 0) {
          sm.P[b ^ 1] = r1.p;
          sm.V[b ^ 1] = r1.V;
        }
      }
      if constexpr (HALF) tcx::cp_async_wait_all();
      tcx::fence_async_smem();
      tile_bar();
      if (tid == 0 && ok) {
        tcx::mbar_arrive(&sm.ready[b]);
        if (next) {
          issue_gram<DW>(A, tmem, &sm.mma);
          ++issued;
        }
      }
      r1 = r2;
      r2 = r3;
      p3 = p4;
    }
  } else {
    bool ok = true;
    unsigned long long rows = 0;
    for (int64_t k = 0; k < NK && ok; ++k) {
      const int b = (int)(k & 1);
      ok = pipe_wait(sm, &sm.ready[b], (uint32_t)((k >> 1) & 1), &ctr->status, lane);
      if (!ok) break;
      const int64_t p = sm.P[b];
      const int ns = gram_sweep<T, !HALF>(list_of(sm, b), sm.S, sm.V[b], Xs, d, dpad, p, ra, lane, ties);
      for (int t = lane; t < J.out_stride; t += 32) J.out[p * J.out_stride + t] = t < ns ? sm.S[t] : -1;
      if (lane == 0) J.out_deg[p] = ns;
      edges += ns;
      ++rows;
      __syncwarp();
      if (lane == 0) tcx::mbar_arrive(&sm.freed[b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
    if (lane == 0) {
      if (ties) atomicAdd(&ctr->rule_ties, ties);
      if (J.merge && rows) {
        atomicAdd(&ctr->merge_repruned, rows);
        atomicAdd(&ctr->edges, edges);
      }
    }
  }
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) {
    // an MMA left outstanding by an expired wait gets one more bounded wait before TMEM is freed
    issued = __shfl_sync(FULL, issued, 0);
    completed = __shfl_sync(FULL, completed, 0);
    if (issued > completed) tcx::mbar_wait_warp(&sm.mma, (issued - 1) & 1u);
    tcx::fence_after();
    tcx::tmem_dealloc<GT_N>(tmem);
  }
}

// ---- K6 lists for the pipelined re-prune --------------------------------------------------------
// Merged set V'(p) = N+(p) U in(p) with exact D(p, .) and its (D, id) order.  |V'| <= R: written
// to adj in that order; R < |V'| <= 128: written to the list rows and p appended to rlist (count
// ctr->nre) for gram_pipe_kernel; larger sets go to mid_list for the 256-entry pass.  No tensor
// memory, so many CTAs per SM hide the chain of dependent loads.
template <int DW>
__global__ void __launch_bounds__(128)
merge_lists_u8_kernel(const uint8_t* __restrict__ U, int64_t n, const int32_t* __restrict__ fwd,
                      const int32_t* __restrict__ fdeg, const int64_t* __restrict__ off,
                      const int32_t* __restrict__ inl, int R, int rs, int32_t* __restrict__ adj,
                      int32_t* __restrict__ deg, int32_t* __restrict__ mlist,
                      float* __restrict__ mdist, int32_t* __restrict__ mlen,
                      int32_t* __restrict__ rlist, int32_t* __restrict__ mid_list, Counters* ctr) {
  __shared__ int32_t s_raw[GT_N];
  __shared__ uint64_t s_key[GT_N];
  __shared__ uint4 s_p[8];
  __shared__ int s_nv;
  const int tid = threadIdx.x;
  unsigned long long edges = 0, maxlist = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    const int nf = fdeg[p];
    const int64_t i0 = off[p];
    const int nin = (int)(off[p + 1] - i0);
    if (nf + nin > GT_N) {  // uniform: deferred to the 256-entry pass
      if (tid == 0) mid_list[atomicAdd(&ctr->nmid, 1)] = (int32_t)p;
      continue;
    }
    maxlist = max(maxlist, (unsigned long long)(nf + nin));
    const int32_t* fp = fwd + p * R;
    if (tid < nf) s_raw[tid] = fp[tid];
    if (tid == 0) s_nv = nf;
    if (tid < DW / 4) s_p[tid] = __ldg(reinterpret_cast<const uint4*>(U + p * (DW * 4)) + tid);
    __syncthreads();
    if (tid < nin) {  // in-neighbours not already in N+(p)
      const int32_t u = inl[i0 + tid];
      bool dup = false;
      for (int k = 0; k < nf && !dup; ++k) dup = fp[k] == u;
      if (!dup) s_raw[atomicAdd(&s_nv, 1)] = u;
    }
    __syncthreads();
    const int V = s_nv;
    uint32_t d2 = 0;
    int32_t u = 0;
    if (tid < V) {
      u = s_raw[tid];
      uint4 w[DW / 4];
      load_row<DW>(U, u, w);
      d2 = row_norm<DW>(w) + row_norm<DW>(s_p) - 2u * row_dot<DW>(w, s_p);
      s_key[tid] = pack_key((float)d2, u);
    }
    __syncthreads();
    if (tid < V) {
      const uint64_t k = s_key[tid];
      int rank = 0;
      for (int q = 0; q < V; ++q) rank += s_key[q] < k;
      if (V <= R) {
        adj[p * rs + rank] = u;
      } else {
        mlist[p * GT_N + rank] = u;
        mdist[p * GT_N + rank] = sqrtf((float)d2);
      }
    }
    if (V <= R) {
      for (int t = V + tid; t < rs; t += blockDim.x) adj[p * rs + t] = -1;
      if (tid == 0) deg[p] = V;
      edges += V;
    } else if (tid == 0) {
      mlen[p] = V;
      rlist[atomicAdd(&ctr->nre, 1)] = (int32_t)p;
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (edges) atomicAdd(&ctr->edges, edges);
    atomicMax(&ctr->merge_max_list, maxlist);
  }
}

// ---- K6, first pass ----------------------------------------------------------------------------
// Merged sets V'(p) = N+(p) U in(p) of up to 128 entries; larger sets go to mid_list for the
// 256-entry SIMT pass.  |V'| <= R: kept in (D, id) order; otherwise pruned once on the Gram tile.
template <typename T, int DW>
__global__ void __launch_bounds__(GT_THREADS)
merge_gram_u8_kernel(const uint8_t* __restrict__ U, const T* __restrict__ Xs, int64_t n, int d,
                     int dpad, const int32_t* __restrict__ fwd, const int32_t* __restrict__ fdeg,
                     const int64_t* __restrict__ off, const int32_t* __restrict__ inl, RuleArgs ra,
                     int32_t* __restrict__ adj, int32_t* __restrict__ deg, Counters* ctr,
                     int32_t* __restrict__ mid_list) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* A = align1024(smem_raw);
  GramSmem& sm = *reinterpret_cast<GramSmem*>(A + GT_ABYTES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  gram_setup(sm, warp);
  const uint32_t tmem = sm.tmem;
  uint32_t phase = 0;
  unsigned long long ties = 0, repruned = 0, edges = 0, maxlist = 0;
  for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
    const int nf = fdeg[p];
    const int64_t i0 = off[p];
    const int nin = (int)(off[p + 1] - i0);
    if (nf + nin > GT_N) {  // uniform: deferred to the 256-entry pass
      if (tid == 0) mid_list[atomicAdd(&ctr->nmid, 1)] = (int32_t)p;
      continue;
    }
    maxlist = max(maxlist, (unsigned long long)(nf + nin));
    const int32_t* fp = fwd + p * ra.R;
    if (tid < nf) sm.raw[tid] = fp[tid];
    if (tid == 0) sm.nv = nf;
    if (tid < DW / 4) sm.prow[tid] = __ldg(reinterpret_cast<const uint4*>(U + p * (DW * 4)) + tid);
    __syncthreads();
    if (tid < nin) {  // in-neighbours not already in N+(p)
      const int32_t u = inl[i0 + tid];
      bool dup = false;
      for (int k = 0; k < nf && !dup; ++k) dup = fp[k] == u;
      if (!dup) sm.raw[atomicAdd(&sm.nv, 1)] = u;
    }
    __syncthreads();
    const int V = sm.nv;
    uint4 w[DW / 4];
    uint32_t d2 = 0, nu = 0;
    int32_t u = 0;
    if (tid < V) {
      u = sm.raw[tid];
      load_row<DW>(U, u, w);
      nu = row_norm<DW>(w);
      const uint32_t np = row_norm<DW>(sm.prow);
      d2 = nu + np - 2u * row_dot<DW>(w, sm.prow);
      sm.key[tid] = pack_key((float)d2, u);
    }
    __syncthreads();
    int rank = 0;
    if (tid < V) {  // rank among the distinct (D, id) keys
      const uint64_t k = sm.key[tid];
      for (int q = 0; q < V; ++q) rank += sm.key[q] < k;
      sm.ids[rank] = u;
      sm.dist[rank] = sqrtf((float)d2);
    }
    int na = V;
    if (V > ra.R) {
      if (tid < V) {
        sm.nrm[rank] = (float)nu;
        store_row_f16<DW>(w, rank, A);
      }
      if (!gram_mma<DW>(sm, A, tmem, phase, &ctr->status, lane)) break;
      int steps;
      na = gram_prune(sm, tmem, V, Xs, d, dpad, p, ra, warp, lane, &ctr->status, ties, &steps);
      ++repruned;
    } else {
      __syncthreads();
      if (tid < V) sm.S[tid] = sm.ids[tid];
      __syncthreads();
    }
    int32_t* row = adj + p * ra.rs;
    for (int t = tid; t < ra.rs; t += GT_THREADS) row[t] = t < na ? sm.S[t] : -1;
    if (tid == 0) deg[p] = na;
    edges += na;
    tcx::fence_before();
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if (lane == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (tid == 0) {
    atomicAdd(&ctr->merge_repruned, repruned);
    atomicAdd(&ctr->edges, edges);
    atomicMax(&ctr->merge_max_list, maxlist);
  }
  gram_teardown(sm, tmem, phase, warp);
}

// ---- K4 for float rows on CUDA cores: all pairs of a list in 32 x 32 blocks ----------------------
// Lists of up to 256 entries (FP32 or FP16 rows of any width, fixed alpha).  A warp computes a
// block of the list's Gram matrix (i in rows 32a..32a+31, j in 32b..32b+31, a <= b): lane l owns
// entry j = 32b + l and accumulates <x_i, x_j> for the 32 rows i, broadcast from shared memory
// in double-buffered chunks of PP_KC dimensions (cp.async), one FFMA per pair and dimension (a
// chain of d); each warp carries two blocks per pass, sharing the row loads when their row
// blocks agree.  With |x|^2 from FP32 chains too,
// D^2 = |x_i|^2 + |x_j|^2 - 2 <x_i, x_j> is off by at most cE (|x_i|^2 + |x_j|^2),
// cE = (2 d + 8) 2^-24 (the |x_ik x_jk| sum to at most the mean of the two squared norms),
// and the rule is decided in the squared form with the certified window of the FP16 Gram tiles;
// open pairs are decided again when Alg. 2 meets them by the FP32 difference form with the band,
// then FP64.  Lane l keeps the 32 decisions of its entry as one word of the "prunes" / "open"
// masks; warp 0 runs Alg. 2 on them.
constexpr int PP_THREADS = 256;
constexpr int PP_VMAX = 256;
constexpr int PP_NW = PP_VMAX / 32;  // mask words per entry
constexpr int PP_KC = 32;            // dimensions per staged chunk
constexpr int PP_LD = PP_KC + 4;     // row stride in floats: rows r..r+7 in distinct bank groups

struct __align__(16) PairsSmem {
  float xs[2][PP_VMAX][PP_LD];  // double-buffered dimension chunks of the list's rows
  int32_t ids[PP_VMAX];
  float dist[PP_VMAX];
  float nrm[PP_VMAX];
  uint32_t bp[PP_VMAX][PP_NW];
  uint32_t bt[PP_VMAX][PP_NW];
  int32_t S[64];
  int ns;
};
constexpr int PP_SMEM = (int)sizeof(PairsSmem);

// Alg. 2 on the all-pairs masks: PP_NW words per entry (V <= 256), near-ties re-decided by the
// FP32 difference form with the band, then FP64.
template <typename T>
CNG_DEV int pairs_sweep(PairsSmem& sm, int V, const T* __restrict__ Xs, int d, int dpad, int64_t p,
                        const RuleArgs& r, int lane, unsigned long long& ties) {
  const GramList gl{sm.ids, sm.dist, sm.nrm, nullptr, nullptr};
  return mask_sweep<T, false, PP_NW / 4>(gl, reinterpret_cast<const uint4*>(sm.bp),
                                         reinterpret_cast<const uint4*>(sm.bt), sm.S, V, Xs, d, dpad, p, r,
                                         lane, ties);
}

// Block t of the blocks (a, b), a <= b < nb, in row-major order (a outer): consecutive blocks
// share their row block a except across row boundaries.
CNG_DEV void block_of(int t, int nb, int& a, int& b) {
  a = 0;
  while (t >= nb - a) {
    t -= nb - a;
    ++a;
  }
  b = a + t;
}

// Four consecutive elements of row `row` from dimension k as floats (zero at k >= d).
CNG_DEV float4 load4(const float* __restrict__ row, int k, int d) {
  if (k + 4 <= d) return __ldg(reinterpret_cast<const float4*>(row + k));
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < d) v.x = row[k];
  if (k + 1 < d) v.y = row[k + 1];
  if (k + 2 < d) v.z = row[k + 2];
  return v;
}
CNG_DEV float4 load4(const __half* __restrict__ row, int k, int d) {
  if (k + 4 <= d) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(row + k));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < d) v.x = __half2float(row[k]);
  if (k + 1 < d) v.y = __half2float(row[k + 1]);
  if (k + 2 < d) v.z = __half2float(row[k + 2]);
  return v;
}

// Dimensions [k0, k0 + PP_KC) of every entry's row into chunk buffer buf: 16-byte cp.async copies
// of the zero-padded stored rows (FP32), or converted loads (FP16).
template <typename T>
CNG_DEV void stage_chunk(PairsSmem& sm, int buf, const T* __restrict__ Xs, int d, int dpad, int V,
                         int k0) {
  for (int e = threadIdx.x; e < V * (PP_KC / 4); e += PP_THREADS) {
    const int i = e / (PP_KC / 4), q = e - i * (PP_KC / 4);
    const T* row = Xs + (int64_t)sm.ids[i] * dpad;
    if constexpr (sizeof(T) == 4) {
      tcx::cp_async16(&sm.xs[buf][i][4 * q], row + k0 + 4 * q);  // k0 + 4q + 4 <= dpad
    } else {
      *reinterpret_cast<float4*>(&sm.xs[buf][i][4 * q]) = load4(row, k0 + 4 * q, d);
    }
  }
  tcx::cp_async_commit();
}

// One job (the GramJob contract): rows q < count, the list of point p = pts[q] (or q) at row p.
template <typename T>
__global__ void __launch_bounds__(PP_THREADS, 2)
pairs_prune_kernel(const T* __restrict__ Xs, int d, int dpad, GramJob J, RuleArgs ra, Counters* ctr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PairsSmem& sm = *reinterpret_cast<PairsSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nchunk = (d + PP_KC - 1) / PP_KC;
  // Gram and norms both FP32 chains of d: cE = (2 d + 8) 2^-24
  const float cE = (float)(2 * d + 8) * 5.9604644775390625e-8f;
  const float A2 = ra.alpha32 * ra.alpha32, A2cE = A2 * cE;
  unsigned long long ties = 0, rows = 0, edges = 0;
  const int64_t nq = J.count ? (int64_t)*J.count : J.n;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const int64_t p = J.pts ? (int64_t)J.pts[q] : q;
    const int V = J.len ? J.len[p] : J.L;
    const int nb = (V + 31) >> 5;
    const int nblocks = nb * (nb + 1) / 2;
    for (int t = tid; t < V; t += PP_THREADS) {
      sm.ids[t] = J.ids[p * J.list_stride + t];
      sm.dist[t] = J.dist[p * J.list_stride + t];
    }
    float nn = 0.f;  // |x_tid|^2 (pass 0)
    // up to 16 blocks per pass over the 8 warps: with P blocks in the pass, the first P - 8
    // warps take two consecutive blocks (row-major order: when they share their row block a,
    // each broadcast row load serves both), the others one
    for (int pass = 0; pass * 16 < nblocks; ++pass) {
      const int P = min(16, nblocks - pass * 16), np = max(0, P - 8);
      const int blk0 = pass * 16 + (warp < np ? 2 * warp : np + warp);
      const int blk1 = warp < np ? blk0 + 1 : nblocks;
      const bool has0 = warp < np || np + warp < P, has1 = warp < np;
      int a0 = 0, b0 = 0, a1 = 0, b1 = 0;
      if (has0) block_of(blk0, nb, a0, b0);
      if (has1) block_of(blk1, nb, a1, b1);
      float acc0[32], acc1[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) acc0[r] = acc1[r] = 0.f;
      __syncthreads();  // ids written; both chunk buffers free
      stage_chunk(sm, 0, Xs, d, dpad, V, 0);
      for (int c = 0; c < nchunk; ++c) {
        const int buf = c & 1;
        if (c + 1 < nchunk) {
          stage_chunk(sm, buf ^ 1, Xs, d, dpad, V, (c + 1) * PP_KC);
          asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
          tcx::cp_async_wait_all();
        }
        __syncthreads();  // chunk c visible to every warp
        if (pass == 0 && tid < V) {
#pragma unroll
          for (int k = 0; k < PP_KC; k += 4) {
            const float4 x = *reinterpret_cast<const float4*>(&sm.xs[buf][tid][k]);
            nn = fmaf(x.x, x.x, nn);
            nn = fmaf(x.y, x.y, nn);
            nn = fmaf(x.z, x.z, nn);
            nn = fmaf(x.w, x.w, nn);
          }
        }
        if (has1 && a1 == a0) {  // shared rows
          const float* xj0 = sm.xs[buf][32 * b0 + lane];
          const float* xj1 = sm.xs[buf][32 * b1 + lane];
#pragma unroll 1
          for (int k = 0; k < PP_KC; k += 4) {
            const float4 y0 = *reinterpret_cast<const float4*>(xj0 + k);
            const float4 y1 = *reinterpret_cast<const float4*>(xj1 + k);
#pragma unroll
            for (int r = 0; r < 32; ++r) {
              const float4 x = *reinterpret_cast<const float4*>(&sm.xs[buf][32 * a0 + r][k]);
              acc0[r] = fmaf(x.x, y0.x, acc0[r]);
              acc1[r] = fmaf(x.x, y1.x, acc1[r]);
              acc0[r] = fmaf(x.y, y0.y, acc0[r]);
              acc1[r] = fmaf(x.y, y1.y, acc1[r]);
              acc0[r] = fmaf(x.z, y0.z, acc0[r]);
              acc1[r] = fmaf(x.z, y1.z, acc1[r]);
              acc0[r] = fmaf(x.w, y0.w, acc0[r]);
              acc1[r] = fmaf(x.w, y1.w, acc1[r]);
            }
          }
        } else if (has0) {
          const float* xj0 = sm.xs[buf][32 * b0 + lane];
          const float* xj1 = sm.xs[buf][32 * b1 + lane];
#pragma unroll 1
          for (int k = 0; k < PP_KC; k += 4) {
            const float4 y0 = *reinterpret_cast<const float4*>(xj0 + k);
#pragma unroll
            for (int r = 0; r < 32; ++r) {
              const float4 x = *reinterpret_cast<const float4*>(&sm.xs[buf][32 * a0 + r][k]);
              acc0[r] = fmaf(x.x, y0.x, acc0[r]);
              acc0[r] = fmaf(x.y, y0.y, acc0[r]);
              acc0[r] = fmaf(x.z, y0.z, acc0[r]);
              acc0[r] = fmaf(x.w, y0.w, acc0[r]);
            }
            if (has1) {
              const float4 y1 = *reinterpret_cast<const float4*>(xj1 + k);
#pragma unroll
              for (int r = 0; r < 32; ++r) {
                const float4 x = *reinterpret_cast<const float4*>(&sm.xs[buf][32 * a1 + r][k]);
                acc1[r] = fmaf(x.x, y1.x, acc1[r]);
                acc1[r] = fmaf(x.y, y1.y, acc1[r]);
                acc1[r] = fmaf(x.z, y1.z, acc1[r]);
                acc1[r] = fmaf(x.w, y1.w, acc1[r]);
              }
            }
          }
        }
        __syncthreads();  // chunk c consumed: its buffer may be refilled
      }
      if (pass == 0 && tid < V) sm.nrm[tid] = nn;
      __syncthreads();  // norms visible
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {  // decisions of the blocks' pairs (i, j), i < j < V
        const bool has = h == 0 ? has0 : has1;
        if (!has) continue;
        const int a = h == 0 ? a0 : a1, b = h == 0 ? b0 : b1;
        const int j = 32 * b + lane;
        if (j >= V) continue;
        const float dj = sm.dist[j], nj = sm.nrm[j];
        const float tj = dj - ra.t32;
        const float lim = 2.f * ra.band * dj;
        const int cls = tj > lim ? 0 : (tj < -lim ? 1 : 2);
        const float T2 = tj * tj, w = 2.f * ra.band * dj * tj;
        uint32_t pb = 0u, tb = 0u;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int i = 32 * a + r;
          const float g = h == 0 ? acc0[r] : acc1[r];
          if (i < j) {
            const float ni = sm.nrm[i];
            const float d2 = (nj - g) + (ni - g);
            const float e = fmaf(-A2, d2, T2);
            const float win =
                fmaf(2.384185791015625e-7f, fmaf(A2, fabsf(d2), T2), fmaf(A2cE, nj + ni, w));
            if (cls == 2 || (cls == 0 && fabsf(e) <= win)) tb |= 1u << r;
            else if (cls == 0 && e > win) pb |= 1u << r;
          }
        }
        sm.bp[j][a] = pb;
        sm.bt[j][a] = tb;
      }
    }
    __syncthreads();
    if (warp == 0) {
      const int k = pairs_sweep(sm, V, Xs, d, dpad, p, ra, lane, ties);
      if (lane == 0) sm.ns = k;
    }
    __syncthreads();
    const int ns = sm.ns;
    for (int t = tid; t < J.out_stride; t += PP_THREADS) J.out[p * J.out_stride + t] = t < ns ? sm.S[t] : -1;
    if (tid == 0) J.out_deg[p] = ns;
    edges += ns;
    ++rows;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ties += __shfl_xor_sync(FULL, ties, o);
  if (lane == 0 && ties) atomicAdd(&ctr->rule_ties, ties);
  if (tid == 0 && J.merge && rows) {
    atomicAdd(&ctr->merge_repruned, rows);
    atomicAdd(&ctr->edges, edges);
  }
}

template <typename K>
static void prepare(K kernel) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM);
}

}  // namespace

bool gram_prune_ok(const uint8_t* U, int dw, int L, int R) {
  return U && L >= 1 && L <= GT_N && R <= 64 && (dw == 8 || dw == 16 || dw == 24 || dw == 32);
}

bool gram_prune_f16_ok(int dtype, int dpad, int L, int R, bool adaptive) {
  return dtype == CNG_F16 && !adaptive && (dpad == 64 || dpad == 128) && L >= 1 && L <= GT_N &&
         R <= 64;
}

// |x|^2 of every FP16 row: FP64 sum of the exact squares, rounded once to FP32.
__global__ void half_norms_kernel(const __half* __restrict__ X, int64_t n, int d, int dpad,
                                  float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const __half* x = X + i * dpad;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      const double v = (double)__half2float(x[k]);
      s = fma(v, v, s);
    }
    out[i] = (float)s;
  }
}

bool pairs_prune_ok(int L, int R, bool adaptive) { return !adaptive && L >= 1 && L <= PP_VMAX && R <= 64; }

static cudaError_t pairs_job(const void* xs, int dtype, int d, int dpad, const GramJob& J,
                             const RuleArgs& ra, Counters* ctr, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(J.n, (int64_t)num_sms() * 2);
  count_launch();
  if (dtype == CNG_F32) {
    cudaFuncSetAttribute(pairs_prune_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, PP_SMEM);
    pairs_prune_kernel<float><<<grid, PP_THREADS, PP_SMEM, s>>>((const float*)xs, d, dpad, J, ra, ctr);
  } else {
    cudaFuncSetAttribute(pairs_prune_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, PP_SMEM);
    pairs_prune_kernel<__half><<<grid, PP_THREADS, PP_SMEM, s>>>((const __half*)xs, d, dpad, J, ra, ctr);
  }
  return cudaGetLastError();
}

cudaError_t launch_prune_pairs(const void* xs, int dtype, int64_t n, int d, int dpad,
                               const int32_t* cand, const float* cdist, int L, const RuleArgs& ra,
                               int32_t* fwd, int32_t* fdeg, Counters* ctr, cudaStream_t s) {
  const GramJob J{cand, cdist, L, nullptr, L, nullptr, nullptr, n, fwd, ra.R, fdeg, 0, nullptr};
  return pairs_job(xs, dtype, d, dpad, J, ra, ctr, s);
}

cudaError_t launch_merge_pairs(const void* xs, int dtype, int64_t n, int d, int dpad,
                               const MergeScratch& ms, const RuleArgs& ra, int32_t* adj, int32_t* deg,
                               Counters* ctr, cudaStream_t s) {
  const GramJob J{ms.mlist, ms.mdist, ms.stride, ms.mlen, 0, ms.rlist, &ctr->nre, n, adj, ra.rs, deg, 1,
                  nullptr};
  return pairs_job(xs, dtype, d, dpad, J, ra, ctr, s);
}

cudaError_t launch_prune_gram_f16(const void* xs, int64_t n, int d, int dpad, const int32_t* cand,
                                  const float* cdist, int L, const RuleArgs& ra, int32_t* fwd,
                                  int32_t* fdeg, float* norms, Counters* ctr, cudaStream_t s) {
  const __half* X = static_cast<const __half*>(xs);
  count_launch();
  half_norms_kernel<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, s>>>(
      X, n, d, dpad, norms);
  const int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 4);
  const GramJob J{cand, cdist, L, nullptr, L, nullptr, nullptr, n, fwd, ra.R, fdeg, 0, norms};
  count_launch();
  if (dpad == 128) {
    prepare(gram_pipe_kernel<__half, 128, true>);
    gram_pipe_kernel<__half, 128, true><<<grid, GP_THREADS, GT_SMEM, s>>>(nullptr, X, d, dpad, J, ra, ctr);
  } else {
    prepare(gram_pipe_kernel<__half, 64, true>);
    gram_pipe_kernel<__half, 64, true><<<grid, GP_THREADS, GT_SMEM, s>>>(nullptr, X, d, dpad, J, ra, ctr);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prune_gram_t(const uint8_t* U, int dw, const T* xs, int64_t n, int d, int dpad,
                                const int32_t* cand, const float* cdist, int L, const RuleArgs& ra,
                                int32_t* fwd, int32_t* fdeg, Counters* ctr, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 4);
  const GramJob J{cand, cdist, L, nullptr, L, nullptr, nullptr, n, fwd, ra.R, fdeg, 0, nullptr};
#define CNG_PG(DW)                                                                                \
  if (dw == DW) {                                                                                 \
    count_launch();                                                                               \
    if (ra.imax < 0) {                                                                            \
      prepare(gram_pipe_kernel<T, 4 * DW, false>);                                                \
      gram_pipe_kernel<T, 4 * DW, false><<<grid, GP_THREADS, GT_SMEM, s>>>(U, xs, d, dpad, J, ra, \
                                                                           ctr);                  \
    } else {                                                                                      \
      prepare(prune_gram_u8_kernel<T, DW>);                                                       \
      prune_gram_u8_kernel<T, DW><<<grid, GT_THREADS, GT_SMEM, s>>>(U, xs, n, d, dpad, cand,      \
                                                                    cdist, L, ra, fwd, fdeg, ctr); \
    }                                                                                             \
    return cudaGetLastError();                                                                    \
  }
  CNG_PG(8)
  CNG_PG(16)
  CNG_PG(24)
  CNG_PG(32)
#undef CNG_PG
  return cudaErrorInvalidValue;
}

cudaError_t launch_prune_gram_u8(const uint8_t* U, int dw, const void* xs, int dtype, int64_t n,
                                 int d, int dpad, const int32_t* cand, const float* cdist, int L,
                                 const RuleArgs& ra, int32_t* fwd, int32_t* fdeg, Counters* ctr,
                                 cudaStream_t s) {
  return dtype == CNG_F32
             ? prune_gram_t(U, dw, (const float*)xs, n, d, dpad, cand, cdist, L, ra, fwd, fdeg, ctr, s)
             : prune_gram_t(U, dw, (const __half*)xs, n, d, dpad, cand, cdist, L, ra, fwd, fdeg, ctr,
                            s);
}

template <typename T>
static cudaError_t merge_gram_t(const uint8_t* U, int dw, const T* xs, int64_t n, int d, int dpad,
                                const int32_t* fwd, const int32_t* fdeg, const int64_t* off,
                                const int32_t* inl, const RuleArgs& ra, int32_t* adj, int32_t* deg,
                                Counters* ctr, int32_t* mid_list, const MergeScratch& ms,
                                cudaStream_t s) {
  const int grid = (int)std::min<int64_t>(n, (int64_t)num_sms() * 4);
  const bool pipe = ra.imax < 0 && ms.mlist;
  const GramJob J{ms.mlist, ms.mdist, ms.stride, ms.mlen, 0, ms.rlist, &ctr->nre, n, adj, ra.rs, deg, 1,
                  nullptr};
  const int glist = (int)std::min<int64_t>(n, (int64_t)num_sms() * 16);
#define CNG_MG(DW)                                                                                 \
  if (dw == DW) {                                                                                  \
    if (pipe) {                                                                                    \
      count_launch();                                                                              \
      merge_lists_u8_kernel<DW><<<glist, 128, 0, s>>>(U, n, fwd, fdeg, off, inl, ra.R, ra.rs, adj,  \
                                                      deg, ms.mlist, ms.mdist, ms.mlen, ms.rlist,  \
                                                      mid_list, ctr);                              \
      prepare(gram_pipe_kernel<T, 4 * DW, false>);                                                 \
      count_launch();                                                                              \
      gram_pipe_kernel<T, 4 * DW, false><<<num_sms() * 4, GP_THREADS, GT_SMEM, s>>>(U, xs, d, dpad, \
                                                                                    J, ra, ctr);   \
    } else {                                                                                       \
      prepare(merge_gram_u8_kernel<T, DW>);                                                        \
      count_launch();                                                                              \
      merge_gram_u8_kernel<T, DW><<<grid, GT_THREADS, GT_SMEM, s>>>(U, xs, n, d, dpad, fwd, fdeg,  \
                                                                    off, inl, ra, adj, deg, ctr,   \
                                                                    mid_list);                     \
    }                                                                                              \
    return cudaGetLastError();                                                                     \
  }
  CNG_MG(8)
  CNG_MG(16)
  CNG_MG(24)
  CNG_MG(32)
#undef CNG_MG
  return cudaErrorInvalidValue;
}

cudaError_t launch_merge_gram_u8(const uint8_t* U, int dw, const void* xs, int dtype, int64_t n,
                                 int d, int dpad, const int32_t* fwd, const int32_t* fdeg,
                                 const int64_t* off, const int32_t* inl, const RuleArgs& ra,
                                 int32_t* adj, int32_t* deg, Counters* ctr, int32_t* mid_list,
                                 const MergeScratch& ms, cudaStream_t s) {
  return dtype == CNG_F32
             ? merge_gram_t(U, dw, (const float*)xs, n, d, dpad, fwd, fdeg, off, inl, ra, adj, deg,
                            ctr, mid_list, ms, s)
             : merge_gram_t(U, dw, (const __half*)xs, n, d, dpad, fwd, fdeg, off, inl, ra, adj, deg,
                            ctr, mid_list, ms, s);
}

}  // namespace cng
