// k_search_fast.cu -- batched beam search of Alg. 1 with each warp's queue in registers, sm_103a.
//
// Data stored as exact 8-bit rows (integer coordinates spanning <= 255, d <= 128) gives every
// squared distance as an exact integer below 2^24, so the queue order of Alg. 1 -- by distance,
// then id -- is decided by integer keys alone.  This kernel keeps a warp's queue Q of up to
// 32 * QS entries in registers, entry 32 s + lane in q[s] of that lane, as 64-bit keys
//   key = D^2 << 32 | id << 1 | explored
// whose unsigned order is the (D^2, id) order (ids are below 2^31); KINF pads the tail.
//
// One hop: the first unexplored entry u* of Q (one ballot per slot); its out-list (prefetched
// during the previous hop when the prediction holds); the visited filter (one compare-and-swap
// per probe); the exact distances of the new points, 8 lanes reading each 128-byte row
// (coalesced) and a transposed butterfly handing each distance to its point's lane; a bitonic
// sort of the batch on 32-bit keys D^2 << 5 | lane (64-bit (D^2, id) keys when two distances
// tie); then the merge of the batch into Q as a single bitonic merge network -- the batch,
// reversed, is folded into the last slot (the half-cleaner of the bitonic sequence
// [Q ascending | batch descending]) and log2(32 QS) compare-exchange levels restore the order;
// entries past L are dropped (Alg. 1's truncation to the L closest).  A hop with more than 32 new points merges them 32 at a time,
// which gives the same queue because truncation keeps the L smallest of the union either way.
//
// The visited filter is lossy only in one direction: a point whose probe slots are all taken is
// reported as possibly seen.  Such a point may already be in Q, so it is looked up there (binary
// search over the registers) and dropped when present; a seen point absent from Q lies beyond
// Q's L-th entry, which never grows, and is cut again by the truncation.
//
// Queries that are not exact (non-integer coordinates, or outside the data's range) are
// appended to a list that the general kernel serves afterwards.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "search_internal.h"
#include "search_device.cuh"

namespace cng {
namespace {

constexpr uint64_t KINF = ~0ull;

CNG_DEV uint64_t rkey(uint32_t d2, int32_t id) {
  return ((uint64_t)d2 << 32) | ((uint64_t)(uint32_t)id << 1);
}
CNG_DEV int32_t rkey_id(uint64_t k) { return (int32_t)((uint32_t)k >> 1); }
CNG_DEV float rkey_d2(uint64_t k) { return (float)(uint32_t)(k >> 32); }
CNG_DEV bool unexplored(uint64_t k) { return k != KINF && !(k & 1); }

// Q entry i (i the same in every lane).
template <int QS>
CNG_DEV uint64_t qget(const uint64_t (&q)[QS], int i) {
  uint64_t v = q[0];
#pragma unroll
  for (int s = 1; s < QS; ++s)
    if ((i >> 5) == s) v = q[s];
  return __shfl_sync(FULL, v, i & 31);
}

// Q entry i (i per lane).
template <int QS>
CNG_DEV uint64_t qget_lane(const uint64_t (&q)[QS], int i) {
  uint64_t r = 0;
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    const uint64_t t = __shfl_sync(FULL, q[s], i & 31);
    if ((i >> 5) == s) r = t;
  }
  return r;
}

// Whether the point of key kb is in Q (binary search on (D^2, id)).
template <int QS>
CNG_DEV bool qcontains(const uint64_t (&q)[QS], uint64_t kb) {
  const uint64_t x = kb >> 1;
  int pos = 0;
#pragma unroll
  for (int step = 16 * QS; step >= 1; step >>= 1)
    if ((qget_lane<QS>(q, pos + step - 1) >> 1) < x) pos += step;
  return (qget_lane<QS>(q, pos) >> 1) == x;
}

// First unexplored entry of Q, or -1 (same in every lane).
template <int QS>
CNG_DEV int first_unexplored(const uint64_t (&q)[QS]) {
  int idx = -1;
#pragma unroll
  for (int s = 0; s < QS; ++s) {
    const unsigned bal = __ballot_sync(FULL, unexplored(q[s]));
    if (idx < 0 && bal) idx = s * 32 + __ffs(bal) - 1;
  }
  return idx;
}

// Q <- the 32 QS smallest of Q and the batch, sorted; kdesc: the batch sorted descending across
// the lanes.  [Q ascending | KINF ... KINF, batch descending] is bitonic; its half-cleaner leaves
// Q unchanged except min(q[QS-1], kdesc), and a bitonic merge of the lower half sorts it.
template <int QS>
CNG_DEV void qmerge(uint64_t (&q)[QS], uint64_t kdesc, int lane) {
  q[QS - 1] = kdesc < q[QS - 1] ? kdesc : q[QS - 1];
#pragma unroll
  for (int st = QS / 2; st >= 1; st >>= 1)
#pragma unroll
    for (int s = 0; s < QS; ++s)
      if (!(s & st)) {
        const uint64_t x = q[s], y = q[s + st];
        q[s] = x < y ? x : y;
        q[s + st] = x < y ? y : x;
      }
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1)
#pragma unroll
    for (int s = 0; s < QS; ++s) {
      const uint64_t o = __shfl_xor_sync(FULL, q[s], j);
      q[s] = (lane & j) ? (o > q[s] ? o : q[s]) : (o < q[s] ? o : q[s]);
    }
}

// Exact squared distances of up to 32 batch rows (row b named by lane b's v, present when
// b < nb), returned in lane b.  G lanes read one row, 16 bytes each, so a warp load covers 32 / G
// whole rows (coalesced) instead of one 16-byte piece of 32 rows; round r of G reads rows
// r * 32 / G + (lane / G).  The G partial sums per lane are reduced across each group by a
// transposed butterfly: after log2(G) exchange levels, lane g of a group holds round g's totals.
// qy: this lane's 16 bytes of the query row (zero past the row, as the stored rows are).
template <int DW>
CNG_DEV uint32_t batch_d2(uint4 qy, const uint8_t* __restrict__ U, int32_t v, int nb, int lane) {
  constexpr int G = DW <= 8 ? 2 : DW <= 16 ? 4 : 8;  // lanes per row
  constexpr int RPR = 32 / G;                         // rows per round
  const int grp = lane / G, g = lane % G;
  uint4 x[G];
#pragma unroll
  for (int r = 0; r < G; ++r) {
    const int b = r * RPR + grp;
    const int32_t vb = __shfl_sync(FULL, v, b);
    x[r] = make_uint4(0u, 0u, 0u, 0u);
    if (b < nb && g * 4 < DW) x[r] = __ldg(reinterpret_cast<const uint4*>(U + (int64_t)vb * (DW * 4)) + g);
  }
  // per byte |x - q| (exact in 8 bits), squared and summed by dp4a
  uint32_t p[G];
#pragma unroll
  for (int r = 0; r < G; ++r) {
    uint32_t t = __vabsdiffu4(x[r].x, qy.x);
    p[r] = __dp4a(t, t, 0u);
    t = __vabsdiffu4(x[r].y, qy.y);
    p[r] = __dp4a(t, t, p[r]);
    t = __vabsdiffu4(x[r].z, qy.z);
    p[r] = __dp4a(t, t, p[r]);
    t = __vabsdiffu4(x[r].w, qy.w);
    p[r] = __dp4a(t, t, p[r]);
  }
#pragma unroll
  for (int s = G / 2; s >= 1; s >>= 1) {  // list length 2 s -> s
    const bool up = g & s;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const uint32_t rv = __shfl_xor_sync(FULL, up ? p[i] : p[i + s], s);
      p[i] = (up ? p[i + s] : p[i]) + rv;
    }
  }
  const uint32_t d2 = p[0];  // row g * RPR + grp
  return __shfl_sync(FULL, d2, (lane % RPR) * G + lane / RPR);
}

// LEARN: the variant that records stop features and runs the stop model (traces and the
// learned mode); the other variant carries none of that state.
template <int DW, int QS, bool LEARN>
__global__ void __launch_bounds__(256, 3) search_fast_kernel(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + (size_t)warp * a.warp_smem_fast;
  uint4* qu = reinterpret_cast<uint4*>(base);                     // query as an 8-bit row
  int32_t* Nv = reinterpret_cast<int32_t*>(base + 128);           // new points of a hop
  float* hist = reinterpret_cast<float*>(Nv + SQ_ROWSLOTS * 32);  // Dk after the last 64 hops
  int32_t* H = reinterpret_cast<int32_t*>(hist + 64);             // visited filter
  StopSmem ms;
  if (LEARN && a.model) {
    unsigned char* mb = smem + (size_t)(blockDim.x >> 5) * a.warp_smem_fast;
    const int4* src = reinterpret_cast<const int4*>(a.model);
    int4* dst = reinterpret_cast<int4*>(mb);
    for (int i = threadIdx.x; i < STOP_BLOCK_BYTES / 16; i += blockDim.x) dst[i] = src[i];
    ms = stop_smem(mb);
    __syncthreads();
  }
  const int hmask = a.hash_slots - 1, L = a.L;
  unsigned long long t_ndc = 0, t_hops = 0, t_stop = 0;

  // each warp takes query (its index) first, then queries nw + (queue head) as it finishes them
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  auto next_item = [&]() -> int64_t {
    int x = 0;
    if (lane == 0) x = atomicAdd(a.counter, 1);
    return nw + __shfl_sync(FULL, x, 0);
  };
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;; it = next_item()) {
    if (it >= a.nq) break;
    const int qi = (int)it;
    if (!a.qids && !(a.qflag && a.qflag[qi] == 0)) {  // not exact: left to the general kernel
      if (lane == 0) a.defer[atomicAdd(a.counter + 1, 1)] = qi;
      continue;
    }
    const uint8_t* src = a.qids ? a.U + (int64_t)a.qids[qi] * (DW * 4) : a.QU + (int64_t)qi * (DW * 4);
    uint32_t qn = 0;
    if (lane < DW / 4) {
      const uint4 x = __ldg(reinterpret_cast<const uint4*>(src) + lane);
      qu[lane] = x;
      qn = __dp4a(x.x, x.x, qn); qn = __dp4a(x.y, x.y, qn);
      qn = __dp4a(x.z, x.z, qn); qn = __dp4a(x.w, x.w, qn);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qn += __shfl_xor_sync(FULL, qn, o);
    for (int c = lane; c < a.hash_slots; c += 32) H[c] = -1;
    __syncwarp();
    constexpr int G = DW <= 8 ? 2 : DW <= 16 ? 4 : 8;  // lanes per row in batch_d2
    const uint4 qy = (lane % G) * 4 < DW ? qu[lane % G] : make_uint4(0u, 0u, 0u, 0u);
    // entry point
    const uint32_t d0 = u8_lane_d2<DW>(qu, qn, a.U, a.entry);
    uint64_t q[QS];
#pragma unroll
    for (int s = 0; s < QS; ++s) q[s] = KINF;
    if (lane == 0) {
      q[0] = rkey(d0, a.entry);
      H[hash32((uint32_t)a.entry) & hmask] = a.entry;
    }
    int len = 1, ndc = 1, hops = 0, flags = 0, tlc = 0;
    const float D0 = sqrtf((float)d0);
    if (lane == 0) hist[0] = D0;
    __syncwarp();
    // every point is explored at most once, so n hops bound a correct search
    const int hop_cap = a.max_hops > 0 ? a.max_hops : (int)min(a.n, (int64_t)0x3fffffff);
    int32_t pf_u = -1;  // predicted next hop vertex and its out-list
    int32_t pf[SQ_ROWSLOTS];
    for (;;) {
      const int idx = first_unexplored<QS>(q);
      if (idx < 0) break;
      if (hops >= hop_cap) {
        flags |= 2;
        if (a.max_hops == 0 && lane == 0) atomicOr(a.status, ST_BOUNDS);
        break;
      }
      const uint64_t ku = qget<QS>(q, idx);
#pragma unroll
      for (int s = 0; s < QS; ++s)
        if (s == (idx >> 5) && lane == (idx & 31)) q[s] |= 1;
      const int32_t u = rkey_id(ku);
      const float Du = sqrtf(rkey_d2(ku));
      ++hops;
      // out-list of u (rows hold -1 past the degree)
      int32_t row[SQ_ROWSLOTS];
      const bool hit = u == pf_u;
#pragma unroll
      for (int r = 0; r < SQ_ROWSLOTS; ++r) {
        const int j = r * 32 + lane;
        row[r] = hit ? pf[r] : (j < a.R ? a.adj[(int64_t)u * a.R + j] : -1);
      }
      // visited filter -> Nv[0 .. nb); bit 31 marks points whose filter slots were full
      int nb = 0;
#pragma unroll
      for (int r = 0; r < SQ_ROWSLOTS; ++r) {
        if (r * 32 >= a.R) break;
        const int32_t v = row[r];
        const int st = v >= 0 ? visit3(H, hmask, v) : 0;
        const unsigned bal = __ballot_sync(FULL, st != 0);
        if (st) Nv[nb + __popc(bal & ((1u << lane) - 1))] = st == 2 ? (int32_t)((uint32_t)v | 0x80000000u) : v;
        nb += __popc(bal);
      }
      __syncwarp();
      ndc += nb;
      bool chg = false;  // the first min(k, |Q|) ids changed
      uint64_t kbs[LEARN ? SQ_ROWSLOTS : 1];  // this hop's sorted batches (stop features)
#pragma unroll
      for (int ci = 0; ci < SQ_ROWSLOTS; ++ci) {
        if constexpr (LEARN) kbs[ci] = KINF;
        if (ci * 32 >= nb) continue;
        const int nbc = min(32, nb - ci * 32);
        const bool has = lane < nbc;
        const int32_t raw = has ? Nv[ci * 32 + lane] : 0;
        const int32_t v = raw & 0x7fffffff;
        const uint32_t d2 = batch_d2<DW>(qy, a.U, v, nbc, lane);
        bool keep = has;
        const bool unsure = has && raw < 0;
        if (__ballot_sync(FULL, unsure)) {  // possibly seen: drop if in Q (or twice in the batch)
          const bool in_q = qcontains<QS>(q, rkey(d2, v));
          const unsigned same = __match_any_sync(FULL, unsure ? v : -1 - lane);
          if (unsure && (in_q || (same & ((1u << lane) - 1)))) keep = false;
        }
        // sort on 32-bit keys D^2 << 5 | lane (D^2 < 2^23 for d <= 128 and a span <= 255), then
        // by id among equal distances
        uint32_t k32 = keep ? (d2 << 5) | (uint32_t)lane : 0xffffffffu;
        k32 = warp_sort32(k32, lane);
        const int32_t vs = __shfl_sync(FULL, v, k32 & 31);
        uint64_t kb = k32 == 0xffffffffu ? KINF : rkey(k32 >> 5, vs);
        const uint32_t prev = __shfl_up_sync(FULL, k32, 1);
        if (__ballot_sync(FULL, lane > 0 && k32 != 0xffffffffu && (prev >> 5) == (k32 >> 5)))
          kb = warp_sort32(kb, lane);
        if constexpr (LEARN) kbs[ci] = kb;
        if (ci == 0) {  // predict the next hop vertex and start loading its out-list
          const int nidx = first_unexplored<QS>(q);
          uint64_t kn = KINF;
          if (nidx >= 0) kn = qget<QS>(q, nidx);
          const uint64_t k0 = __shfl_sync(FULL, kb, 0);
          if (k0 < kn) kn = k0;
          pf_u = kn == KINF ? -1 : rkey_id(kn);
          if (pf_u >= 0) {
#pragma unroll
            for (int r = 0; r < SQ_ROWSLOTS; ++r) {
              const int j = r * 32 + lane;
              pf[r] = j < a.R ? a.adj[(int64_t)pf_u * a.R + j] : -1;
            }
          }
        }
        const int nv = __popc(__ballot_sync(FULL, kb != KINF));
        if (nv == 0) continue;
        const int old_len = len;
        const uint64_t old_kth = old_len >= a.k ? qget<QS>(q, a.k - 1) : 0;
        qmerge<QS>(q, __shfl_sync(FULL, kb, 31 - lane), lane);
        len = min(len + nv, L);
#pragma unroll
        for (int s = 0; s < QS; ++s)
          if (s * 32 + lane >= L) q[s] = KINF;
        // a new point lands in the first k: when |Q| < k its smallest does; otherwise the old
        // k-th entry moves down
        if (old_len < a.k) chg = true;
        else chg |= (qget<QS>(q, a.k - 1) >> 1) != (old_kth >> 1);
      }
      // ---- search state after this hop (learned early stop) ----
      if constexpr (LEARN) {
        const int kk = min(a.k, len);
        const float Dk = sqrtf(rkey_d2(qget<QS>(q, kk - 1)));
        if (chg) tlc = hops;
        const bool want_trace = a.trace_feats && hops <= a.max_trace;
        const bool want_check =
            a.model && (hops % a.check_every) == 0 && hops - tlc >= a.min_stable;
        float f = 0.f;
        if (want_trace || want_check) {
          // points of this hop still in Q: those not beyond its last entry
          int ins = 0;
          const uint64_t last = qget<QS>(q, len - 1);
#pragma unroll
          for (int ci = 0; ci < SQ_ROWSLOTS; ++ci)
            ins += __popc(__ballot_sync(FULL, kbs[ci] != KINF && kbs[ci] <= last));
          int U = 0;
#pragma unroll
          for (int s = 0; s < QS; ++s) U += __popc(__ballot_sync(FULL, unexplored(q[s])));
          const float D1 = sqrtf(rkey_d2(qget<QS>(q, 0)));
          const float DL = sqrtf(rkey_d2(qget<QS>(q, len - 1)));
          f = stop_feature(lane, D0, D1, Dk, DL, Du, hist, hops, tlc, U, len, ins, a.L, a.R);
          if (want_trace && lane < 16)
            a.trace_feats[((int64_t)qi * a.max_trace + (hops - 1)) * 16 + lane] = f;
        }
        __syncwarp();
        if (lane == 0) hist[hops & 63] = Dk;
        __syncwarp();
        if (want_check && mlp_logit(ms, f, lane) >= a.zthr) {
          flags |= 4;
          ++t_stop;
          break;
        }
      }
    }
    // results
#pragma unroll
    for (int s = 0; s < QS; ++s) {
      const int t = s * 32 + lane;
      if (t < a.k) {
        const bool ok = t < len;
        a.ids[(int64_t)qi * a.k + t] = ok ? rkey_id(q[s]) : -1;
        a.dists[(int64_t)qi * a.k + t] = ok ? sqrtf(rkey_d2(q[s])) : INFINITY;
      }
    }
    if (lane == 0) {
      if (a.ndc) a.ndc[qi] = ndc;
      if (a.hops) a.hops[qi] = hops;
      if (a.flags) a.flags[qi] = flags;
      if (a.tlc) a.tlc[qi] = tlc;
    }
    t_ndc += ndc;
    t_hops += hops;
    __syncwarp();
  }
  if (lane == 0) {
    atomicAdd(&a.tot[0], t_ndc);
    atomicAdd(&a.tot[1], t_hops);
    if (t_stop) atomicAdd(&a.tot[3], t_stop);
  }
}

template <int DW, int QS>
cudaError_t launch_fast_t(const SearchArgs& a, int wpb, int grid, cudaStream_t s) {
  const size_t sh = (size_t)wpb * a.warp_smem_fast + (a.model ? STOP_BLOCK_BYTES : 0);
  count_launch();
  if (a.model || a.trace_feats)
    search_fast_kernel<DW, QS, true><<<grid, wpb * 32, sh, s>>>(a);
  else
    search_fast_kernel<DW, QS, false><<<grid, wpb * 32, sh, s>>>(a);
  return cudaGetLastError();
}

template <int DW>
cudaError_t launch_fast_dw(const SearchArgs& a, int qs, int wpb, int grid, cudaStream_t s) {
  switch (qs) {
    case 1: return launch_fast_t<DW, 1>(a, wpb, grid, s);
    case 2: return launch_fast_t<DW, 2>(a, wpb, grid, s);
    case 4: return launch_fast_t<DW, 4>(a, wpb, grid, s);
    case 8: return launch_fast_t<DW, 8>(a, wpb, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int DW, int QS, bool LEARN>
int bps_fast_t(int wpb, size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(search_fast_kernel<DW, QS, LEARN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_fast_kernel<DW, QS, LEARN>, wpb * 32, smem);
  return nb;
}

template <int DW, bool LEARN>
int bps_fast_dw(int qs, int wpb, size_t smem) {
  switch (qs) {
    case 1: return bps_fast_t<DW, 1, LEARN>(wpb, smem);
    case 2: return bps_fast_t<DW, 2, LEARN>(wpb, smem);
    case 4: return bps_fast_t<DW, 4, LEARN>(wpb, smem);
    case 8: return bps_fast_t<DW, 8, LEARN>(wpb, smem);
    default: return 0;
  }
}

template <int DW>
int bps_fast_dw(int qs, bool learn, int wpb, size_t smem) {
  return learn ? bps_fast_dw<DW, true>(qs, wpb, smem) : bps_fast_dw<DW, false>(qs, wpb, smem);
}

}  // namespace

size_t search_fast_warp_smem(int u8w, int hash_slots) {
  (void)u8w;  // the query row takes 128 bytes for every width
  return 128 + SQ_ROWSLOTS * 32 * 4 + 64 * 4 + (size_t)hash_slots * 4;
}

cudaError_t launch_search_fast(const SearchArgs& a, int qs, int wpb, int grid, cudaStream_t s) {
  switch (a.u8w) {
    case 8: return launch_fast_dw<8>(a, qs, wpb, grid, s);
    case 16: return launch_fast_dw<16>(a, qs, wpb, grid, s);
    case 24: return launch_fast_dw<24>(a, qs, wpb, grid, s);
    case 32: return launch_fast_dw<32>(a, qs, wpb, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int search_fast_blocks_per_sm(int u8w, int qs, bool learn, int wpb, size_t smem) {
  switch (u8w) {
    case 8: return bps_fast_dw<8>(qs, learn, wpb, smem);
    case 16: return bps_fast_dw<16>(qs, learn, wpb, smem);
    case 24: return bps_fast_dw<24>(qs, learn, wpb, smem);
    case 32: return bps_fast_dw<32>(qs, learn, wpb, smem);
    default: return 0;
  }
}

}  // namespace cng
