// k_search.cu -- batched beam search of Alg. 1 (K7), general kernel, sm_103a.
//
// One persistent launch serves the batch: each warp takes the next query from an atomic
// counter and runs Alg. 1 to completion; queries of any length share the launch.  On data with
// exact 8-bit rows the register-queue kernel (k_search_fast.cu) runs first and this kernel only
// serves the queries it deferred (non-integer or out-of-range coordinates).
//
// Per warp (shared memory):
//   Q   sorted queue of <= L entries: key = (FP32 squared distance, id), an explored flag,
//       and the canonical FP64 distance when one was needed (NaN otherwise)
//   H   lossy visited filter (open addressing, <= 8 probes); a point missed by the filter is
//       recomputed, then dropped by an exact key match against Q -- or it cannot re-enter Q,
//       because a point that left Q is farther than Q's L-th entry, which never grows
//   q   the query vector
// One hop: first unexplored entry u* of Q (ballot), its out-list (one coalesced load), filter,
// FP32 distances by 8-lane groups (16-byte vector loads), sort of the new batch, merge with
// Q by merge-path ranks (binary search of each side in the other), truncation to L.
//
// Exactness: every comparison whose two FP32 squared distances are within the relative band
// is decided by the canonical FP64 distance and id instead, so the queue order -- and with it
// every hop, the returned ids and the hop count -- equals the FP64 definition of Alg. 1.
// Integer data whose squared distances are exact in FP32 needs no FP64 at all.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "search_internal.h"
#include "search_device.cuh"

namespace cng {

constexpr int SQ_G = 8;
constexpr int SQ_MAXB = 128;  // batch capacity (row stride <= 128)

struct QEnt {
  uint64_t* k;   // keys
  double* x;     // FP64 distance or NaN
  uint8_t* e;    // explored
};

CNG_DEV bool has64(double v) { return !isnan(v); }

// Exact-order comparison: a before b.
CNG_DEV bool before(uint64_t ka, double xa, uint64_t kb, double xb, float band, int exact) {
  if (!exact) {
    float da = key_dist(ka), db = key_dist(kb);
    if (near_tie(da, db, band) && has64(xa) && has64(xb))
      return xa < xb || (xa == xb && key_id(ka) < key_id(kb));
  }
  return ka < kb;
}

template <typename T>
CNG_DEV double canon_q(const float* __restrict__ q, const T* __restrict__ x, int d) {
  return canon_dist(q, x, d);
}

// Squared distance of the query to row v by an 8-lane group, every lane of the group gets it.
// DW == 0: FP32 direct differences over the stored row; DW > 0: exact integer arithmetic on
// 8-bit rows, |q|^2 + |v|^2 - 2 <q, v> (every term below 2^24, so the FP32 value is exact).
template <typename T, int DW>
CNG_DEV float group_sqdist(const float* qv, const uint4* qu, uint32_t qn, const SearchArgs& a,
                           const T* X, int64_t v, int g) {
  if constexpr (DW == 0) {
    float s = part_sqdist<SQ_G>(qv, X + v * a.dpad, a.dpad, g);
    return group_reduce<SQ_G>(s);
  } else {
    uint32_t dot = 0, nv = 0;
    const uint4* r = reinterpret_cast<const uint4*>(a.U + v * (DW * 4));
#pragma unroll
    for (int w = g; w < DW / 4; w += SQ_G) {
      const uint4 x = __ldg(r + w), y = qu[w];
      dot = __dp4a(x.x, y.x, dot); dot = __dp4a(x.y, y.y, dot);
      dot = __dp4a(x.z, y.z, dot); dot = __dp4a(x.w, y.w, dot);
      nv = __dp4a(x.x, x.x, nv); nv = __dp4a(x.y, x.y, nv);
      nv = __dp4a(x.z, x.z, nv); nv = __dp4a(x.w, x.w, nv);
    }
#pragma unroll
    for (int o = SQ_G / 2; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(FULL, dot, o);
      nv += __shfl_xor_sync(FULL, nv, o);
    }
    return (float)(qn + nv - 2u * dot);
  }
}

template <typename T, int DW>
__global__ void __launch_bounds__(256, 4)
search_kernel(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwork = a.qlist ? (int64_t)*a.nq_dev : a.nq;
  if (nwork == 0) return;  // nothing deferred (uniform over the grid)
  const int L = a.L, dpad = a.dpad;
  unsigned char* base = smem + (size_t)warp * a.warp_smem;
  float* qv = reinterpret_cast<float*>(base);
  uint64_t* Ak = reinterpret_cast<uint64_t*>(base + dpad * 4);
  uint64_t* Bk = Ak + L;
  double* Ax = reinterpret_cast<double*>(Bk + L);
  double* Bx = Ax + L;
  uint64_t* Nk = reinterpret_cast<uint64_t*>(Bx + L);
  double* Nx = reinterpret_cast<double*>(Nk + SQ_MAXB);
  int32_t* H = reinterpret_cast<int32_t*>(Nx + SQ_MAXB);
  const int L16 = ((L + 15) / 16) * 16;
  uint8_t* Ae = reinterpret_cast<uint8_t*>(H + a.hash_slots);
  uint8_t* Be = Ae + L16;
  int32_t* Nv = reinterpret_cast<int32_t*>(Be + L16);
  float* hist = reinterpret_cast<float*>(Nv + SQ_MAXB);  // Dk after each of the last 64 hops
  // stop model (shared by the CTA's warps), after all warp regions
  StopSmem ms;
  if (a.model) {
    unsigned char* mb = smem + (size_t)(blockDim.x >> 5) * a.warp_smem;
    const int4* src = reinterpret_cast<const int4*>(a.model);
    int4* dst = reinterpret_cast<int4*>(mb);
    for (int i = threadIdx.x; i < STOP_BLOCK_BYTES / 16; i += blockDim.x) dst[i] = src[i];
    ms = stop_smem(mb);
    __syncthreads();
  }
  const int hmask = a.hash_slots - 1;
  const T* X = reinterpret_cast<const T*>(a.X);
  const int g = lane % SQ_G, grp = lane / SQ_G;
  unsigned long long t_ndc = 0, t_hops = 0, t_f64 = 0, t_stop = 0;

  // work list: all queries, or the ones the register-queue kernel deferred; each warp takes
  // item (its index) first, then items nw + (queue head) as it finishes them
  int* const head = a.qlist ? a.counter + 2 : a.counter;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  auto next_item = [&]() -> int64_t {
    int x = 0;
    if (lane == 0) x = atomicAdd(head, 1);
    return nw + __shfl_sync(FULL, x, 0);
  };
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;; it = next_item()) {
    if (it >= nwork) break;
    int qi = (int)it;
    if (a.qlist) qi = a.qlist[qi];
    // exact queries: the data's FP32 squared distances are exact integers and this query is an
    // integer vector inside the data's range (stored points always are); others resolve
    // near-ties in FP64
    const int qexact = a.exact && (a.qids != nullptr || (a.qflag && a.qflag[qi] == 0));
    const bool use8 = DW > 0 && qexact;
    uint32_t qn = 0;
    if (use8) {  // the query as an 8-bit row in shared memory, and |q|^2
      uint4* qu = reinterpret_cast<uint4*>(qv);
      const uint8_t* src = a.qids ? a.U + (int64_t)a.qids[qi] * (DW * 4) : a.QU + (int64_t)qi * (DW * 4);
      if (lane < DW / 4) {
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(src) + lane);
        qu[lane] = x;
        qn = __dp4a(x.x, x.x, qn); qn = __dp4a(x.y, x.y, qn);
        qn = __dp4a(x.z, x.z, qn); qn = __dp4a(x.w, x.w, qn);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) qn += __shfl_xor_sync(FULL, qn, o);
    } else if (a.qids) {  // the query is a stored point (phase-4 searches)
      load_row(qv, X + (int64_t)a.qids[qi] * dpad, dpad, lane, 32);
    } else {
      const float* qg = a.Q + (int64_t)qi * a.d;
      for (int c = lane; c < dpad; c += 32) qv[c] = c < a.d ? qg[c] : 0.f;
    }
    const uint4* qu = reinterpret_cast<const uint4*>(qv);
    for (int c = lane; c < a.hash_slots; c += 32) H[c] = -1;
    __syncwarp();
    QEnt cur{Ak, Ax, Ae}, nxt{Bk, Bx, Be};
    // entry point
    {
      __syncwarp();
      const float s = use8 ? group_sqdist<T, DW>(qv, qu, qn, a, X, a.entry, g)
                           : group_sqdist<T, 0>(qv, qu, qn, a, X, a.entry, g);
      if (lane == 0) {
        cur.k[0] = pack_key(s, a.entry);
        cur.x[0] = __longlong_as_double(0x7ff8000000000000ll);
        cur.e[0] = 0;
        H[hash32((uint32_t)a.entry) & hmask] = a.entry;
      }
    }
    __syncwarp();
    int len = 1, ndc = 1, hops = 0, flags = 0, tlc = 0;
    const float D0 = sqrtf(key_dist(cur.k[0]));
    if (lane == 0) hist[0] = D0;
    __syncwarp();
    // every point is explored at most once, so n hops bound a correct search; the cap keeps a
    // corrupted queue from looping
    const int hop_cap = a.max_hops > 0 ? a.max_hops : (int)min(a.n, (int64_t)0x3fffffff);
    // adjacency row of the predicted next hop vertex, loaded during the previous hop's merge
    // (used only if the prediction holds; rows have at most SQ_ROWSLOTS * 32 slots)
    int32_t pf_u = -1;
    int32_t pf[SQ_ROWSLOTS];
    for (;;) {
      // first unexplored
      int idx = -1;
      for (int b = 0; b < len && idx < 0; b += 32) {
        int t = b + lane;
        unsigned bal = __ballot_sync(FULL, t < len && !cur.e[t]);
        if (bal) idx = b + __ffs(bal) - 1;
      }
      if (idx < 0) break;
      if (hops >= hop_cap) {
        flags |= 2;
        if (a.max_hops == 0 && lane == 0) atomicOr(a.status, ST_BOUNDS);
        break;
      }
      const int32_t u = key_id(cur.k[idx]);
      const float Du = sqrtf(key_dist(cur.k[idx]));  // distance of the hop vertex
      __syncwarp();
      if (lane == 0) cur.e[idx] = 1;
      ++hops;
      int ins = 0;          // points of this hop still in Q after it
      bool chg = false;     // the first min(k, |Q|) ids changed
      // rows wider than SQ_ROWSLOTS * 32 (a K-NN graph as G0) are taken in slices, each merged
      // into Q before the next: Q keeps the L smallest of everything inserted, whatever the
      // grouping, so the hop's result is Alg. 1's
      for (int rc = 0; rc < a.R; rc += SQ_ROWSLOTS * 32) {
      // fresh neighbours -> Nv[0..nb); rows hold -1 past the degree, so the row alone is read
      int32_t row[SQ_ROWSLOTS];
      const bool hit = rc == 0 && u == pf_u;
#pragma unroll
      for (int r = 0; r < SQ_ROWSLOTS; ++r) {
        const int j = rc + r * 32 + lane;
        row[r] = hit ? pf[r] : (j < a.R ? a.adj[(int64_t)u * a.R + j] : -1);
      }
      int nb = 0;
#pragma unroll
      for (int r = 0; r < SQ_ROWSLOTS; ++r) {
        const int32_t v = row[r];
        bool fresh = v >= 0 && visit(H, hmask, v);
        unsigned bal = __ballot_sync(FULL, fresh);
        if (fresh) Nv[nb + __popc(bal & ((1u << lane) - 1))] = v;
        nb += __popc(bal);
      }
      __syncwarp();
      ndc += nb;
      do {                  // merge of the hop's new points (skipped when there are none)
      if (nb == 0) break;
      int P2;
      bool sorted = false;
      if constexpr (DW > 0) {
        if (use8 && nb <= 32) {  // one lane per neighbour, keys sorted in registers
          uint64_t key = ~0ull;
          if (lane < nb) {
            const int32_t v = Nv[lane];
            key = pack_key(u8_lane_sqdist<DW>(qu, qn, a.U, v), v);
          }
          key = warp_sort32(key, lane);
          Nk[lane] = key;
          Nx[lane] = __longlong_as_double(0x7ff8000000000000ll);
          P2 = 32;
          sorted = true;
          __syncwarp();
        }
      }
      if (!sorted) {
      // FP32 distances, 4 per round
      for (int b0 = 0; b0 < nb; b0 += 32 / SQ_G) {
        int b = b0 + grp;
        int32_t v = b < nb ? Nv[b] : 0;
        const float s = use8 ? group_sqdist<T, DW>(qv, qu, qn, a, X, v, g)
                             : group_sqdist<T, 0>(qv, qu, qn, a, X, v, g);
        if (b < nb && g == 0) {
          Nk[b] = pack_key(s, v);
          Nx[b] = __longlong_as_double(0x7ff8000000000000ll);
        }
      }
      P2 = nb <= 32 ? 32 : (nb <= 64 ? 64 : 128);
      for (int b = nb + lane; b < P2; b += 32) {
        Nk[b] = ~0ull;
        Nx[b] = __longlong_as_double(0x7ff8000000000000ll);
      }
      __syncwarp();
      // sort the batch by FP32 key (bitonic)
      for (int kk = 2; kk <= P2; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < P2; i += 32) {
            int ixj = i ^ j;
            if (ixj > i) {
              uint64_t x0 = Nk[i], y0 = Nk[ixj];
              bool up = (i & kk) == 0;
              if ((x0 > y0) == up) { Nk[i] = y0; Nk[ixj] = x0; }
            }
          }
          __syncwarp();
        }
      }  // !sorted
      {  // predict the next hop vertex (old queue's next unexplored vs the batch's minimum) and
         // start loading its adjacency row
        int nidx = -1;
        for (int b = 0; b < len && nidx < 0; b += 32) {
          const int t = b + lane;
          const unsigned bal = __ballot_sync(FULL, t < len && !cur.e[t]);
          if (bal) nidx = b + __ffs(bal) - 1;
        }
        uint64_t kn = nidx >= 0 ? cur.k[nidx] : ~0ull;
        if (Nk[0] < kn) kn = Nk[0];
        pf_u = kn == ~0ull || a.R > SQ_ROWSLOTS * 32 ? -1 : key_id(kn);
        if (pf_u >= 0) {
#pragma unroll
          for (int r = 0; r < SQ_ROWSLOTS; ++r) {
            const int j = r * 32 + lane;
            pf[r] = j < a.R ? a.adj[(int64_t)pf_u * a.R + j] : -1;
          }
        }
      }
      // drop batch entries already in Q (exact key match; only when the filter lost them)
      int nbv = nb;
      for (int b = lane; b < nb; b += 32) {
        uint64_t kb = Nk[b];
        int lo = 0, hi = len;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (cur.k[mid] < kb) lo = mid + 1; else hi = mid;
        }
        // Q is in exact order, FP32 keys are near-sorted: scan the neighbourhood for equality
        bool dup = false;
        if (qexact) {
          dup = lo < len && cur.k[lo] == kb;
        } else {
          // Q is in exact order, its FP32 keys sorted up to near-ties: scan the window of
          // entries whose FP32 distance lies within four bands of this one
          const float db = key_dist(kb);
          const float lo_d = db * (1.f - 4.f * a.band), hi_d = db * (1.f + 4.f * a.band);
          int l2 = 0, h2 = len;
          while (l2 < h2) {
            int mid = (l2 + h2) >> 1;
            if (key_dist(cur.k[mid]) < lo_d) l2 = mid + 1; else h2 = mid;
          }
          for (int t = l2; t < len && !dup; ++t) {
            if (key_dist(cur.k[t]) > hi_d) break;
            dup = cur.k[t] == kb;
          }
        }
        if (dup) Nk[b] = ~0ull;
      }
      __syncwarp();
      {
        // compact survivors to the front keeping order
        uint64_t kv[SQ_MAXB / 32];
        bool keep[SQ_MAXB / 32];
        int cnt_before = 0;
#pragma unroll
        for (int r = 0; r < SQ_MAXB / 32; ++r) {
          int b = r * 32 + lane;
          kv[r] = b < nb ? Nk[b] : ~0ull;
          keep[r] = b < nb && kv[r] != ~0ull;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < SQ_MAXB / 32; ++r) {
          unsigned bal = __ballot_sync(FULL, keep[r]);
          if (keep[r]) Nk[cnt_before + __popc(bal & ((1u << lane) - 1))] = kv[r];
          cnt_before += __popc(bal);
        }
        nbv = cnt_before;
        __syncwarp();
        for (int b = nbv + lane; b < P2; b += 32) Nk[b] = ~0ull;
        __syncwarp();
      }
      if (nbv == 0) break;
      // near-ties: mark batch entries close to a neighbour in the batch or to a Q entry, and
      // the Q entries concerned; give every marked entry its canonical FP64 distance
      if (!qexact) {
        bool any = false;
        for (int b = lane; b < nbv; b += 32) {
          const float db = key_dist(Nk[b]);
          bool mark = (b > 0 && near_tie(key_dist(Nk[b - 1]), db, a.band)) ||
                      (b + 1 < nbv && near_tie(key_dist(Nk[b + 1]), db, a.band));
          // Q entries within the band: Q keys are sorted up to near-ties; a linear scan of
          // the window found by binary search on FP32 distance covers them
          const float lo_d = db * (1.f - 4.f * a.band), hi_d = db * (1.f + 4.f * a.band);
          int lo = 0, hi = len;
          while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (key_dist(cur.k[mid]) < lo_d) lo = mid + 1; else hi = mid;
          }
          for (int t = lo; t < len; ++t) {
            const float dq = key_dist(cur.k[t]);
            if (dq > hi_d) break;
            if (near_tie(dq, db, a.band)) {
              mark = true;
              if (!has64(cur.x[t]))
                cur.x[t] = canon_q(qv, X + (int64_t)key_id(cur.k[t]) * dpad, a.d);
            }
          }
          if (mark) {
            Nx[b] = canon_q(qv, X + (int64_t)key_id(Nk[b]) * dpad, a.d);
            any = true;
          }
        }
        unsigned anyb = __ballot_sync(FULL, any);
        __syncwarp();
        if (anyb) {
          flags |= 1;
          t_f64 += __popc(anyb);
          // exact re-sort of the batch (odd-even transposition over nbv <= 64)
          for (int ph = 0; ph < nbv; ++ph) {
            for (int b = 2 * lane + (ph & 1); b + 1 < nbv; b += 64) {
              if (before(Nk[b + 1], Nx[b + 1], Nk[b], Nx[b], a.band, 0)) {
                uint64_t tk = Nk[b]; Nk[b] = Nk[b + 1]; Nk[b + 1] = tk;
                double tx = Nx[b]; Nx[b] = Nx[b + 1]; Nx[b + 1] = tx;
              }
            }
            __syncwarp();
          }
        }
      }
      // merge: ranks by binary search of each side in the other (exact comparator)
      const int nlen = min(len + nbv, L);
      for (int i = lane; i < len; i += 32) {
        uint64_t ki = cur.k[i];
        double xi = cur.x[i];
        int lo = 0, hi = nbv;  // # batch entries before Q[i]
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (before(Nk[mid], Nx[mid], ki, xi, a.band, qexact)) lo = mid + 1; else hi = mid;
        }
        int pos = i + lo;
        if (pos < nlen) { nxt.k[pos] = ki; nxt.x[pos] = xi; nxt.e[pos] = cur.e[i]; }
      }
      const int ktop = min(a.k, nlen);
      bool lchg = false;
      int lins = 0;
      for (int b = lane; b < nbv; b += 32) {
        uint64_t kb = Nk[b];
        double xb = Nx[b];
        int lo = 0, hi = len;  // # Q entries before batch[b]
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (before(cur.k[mid], cur.x[mid], kb, xb, a.band, qexact)) lo = mid + 1; else hi = mid;
        }
        int pos = b + lo;
        if (pos < nlen) {
          nxt.k[pos] = kb; nxt.x[pos] = xb; nxt.e[pos] = 0;
          ++lins;
          lchg |= pos < ktop;
        }
      }
      chg = chg || __any_sync(FULL, lchg);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lins += __shfl_xor_sync(FULL, lins, o);
      ins = lins;  // one slice per hop whenever features are recorded (row stride <= 96)
      __syncwarp();
      QEnt t = cur; cur = nxt; nxt = t;
      len = nlen;
      } while (0);
      }  // row slices
      // ---- search state after this hop (learned early stop) ----
      if (a.trace_feats || a.model) {
        const int kk = min(a.k, len);
        const float Dk = sqrtf(key_dist(cur.k[kk - 1]));
        if (chg) tlc = hops;
        const bool want_trace = a.trace_feats && hops <= a.max_trace;
        const bool want_check =
            a.model && (hops % a.check_every) == 0 && hops - tlc >= a.min_stable;
        float f = 0.f;
        if (want_trace || want_check) {
          int U = 0;
          for (int b = 0; b < len; b += 32)
            U += __popc(__ballot_sync(FULL, b + lane < len && !cur.e[b + lane]));
          f = stop_feature(lane, D0, sqrtf(key_dist(cur.k[0])), Dk,
                           sqrtf(key_dist(cur.k[len - 1])), Du, hist, hops, tlc, U, len, ins,
                           a.L, a.R);
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
    for (int t = lane; t < a.k; t += 32) {
      bool ok = t < len;
      a.ids[(int64_t)qi * a.k + t] = ok ? key_id(cur.k[t]) : -1;
      a.dists[(int64_t)qi * a.k + t] = ok ? sqrtf(key_dist(cur.k[t])) : INFINITY;
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
  }
  // t_f64 counts the same warp-wide ballots in every lane
  if (lane == 0) {
    if (t_f64) atomicAdd(&a.tot[2], t_f64);
    if (t_stop) atomicAdd(&a.tot[3], t_stop);
  }
}

size_t search_warp_smem(int dpad, int L, int hash_slots) {
  size_t b = (size_t)dpad * 4 + 4 * (size_t)L * 8 + 2 * SQ_MAXB * 8 + (size_t)hash_slots * 4 +
             2 * (((size_t)L + 15) / 16) * 16 + SQ_MAXB * 4 + 64 * 4;
  return (b + 15) / 16 * 16;
}

template <typename T, int DW>
static cudaError_t launch_general_t(const SearchArgs& a, int warps_per_block, int grid,
                                   cudaStream_t s) {
  const size_t sh = (size_t)warps_per_block * a.warp_smem + (a.model ? STOP_BLOCK_BYTES : 0);
  count_launch();
  search_kernel<T, DW><<<grid, warps_per_block * 32, sh, s>>>(a);
  return cudaGetLastError();
}

// The kernel's shared-memory attribute is set by search_blocks_per_sm (same dtype and u8w),
// which callers run first, outside any stream capture.
cudaError_t launch_search_general(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t s) {
  if (a.dtype != CNG_F32) return launch_general_t<__half, 0>(a, warps_per_block, grid, s);
  switch (a.U ? a.u8w : 0) {
    case 8: return launch_general_t<float, 8>(a, warps_per_block, grid, s);
    case 16: return launch_general_t<float, 16>(a, warps_per_block, grid, s);
    case 24: return launch_general_t<float, 24>(a, warps_per_block, grid, s);
    case 32: return launch_general_t<float, 32>(a, warps_per_block, grid, s);
    default: return launch_general_t<float, 0>(a, warps_per_block, grid, s);
  }
}

bool search_plan(SearchArgs& a, int wpb, int hash_slots, SearchPlan* p) {
  constexpr size_t kMaxBlockSmem = 200 * 1024;
  const size_t extra_smem = a.model ? STOP_BLOCK_BYTES : 0;
  *p = SearchPlan{};
  a.hash_slots = hash_slots;
  a.warp_smem = search_warp_smem(a.dpad, a.L, hash_slots);
  a.warp_smem_fast = 0;
  // the register-queue kernel: exact data with 8-bit rows, L <= 256, and row stride <= 96
  int qs = 0;
  if (a.U && a.exact && a.dtype == CNG_F32 && a.R <= SQ_ROWSLOTS * 32 && a.k <= a.L)
    qs = a.L <= 32 ? 1 : a.L <= 64 ? 2 : a.L <= 128 ? 4 : a.L <= 256 ? 8 : 0;
  if (qs) {
    a.warp_smem_fast = search_fast_warp_smem(a.u8w, hash_slots);
    const size_t sh = (size_t)wpb * a.warp_smem_fast + extra_smem;
    const int b = sh <= kMaxBlockSmem ? search_fast_blocks_per_sm(a.u8w, qs, a.model || a.trace_feats, wpb, sh) : 0;
    if (b < 1) return false;
    p->grid = num_sms() * b;
    p->fast_qs = qs;
  }
  // the general kernel: every query, or the deferred ones (same warps per block when it fits)
  int w = wpb;
  int b = 0;
  for (; w >= 1; w >>= 1) {
    const size_t sh = (size_t)w * a.warp_smem + extra_smem;
    b = sh <= kMaxBlockSmem ? search_blocks_per_sm(a.dtype, a.U ? a.u8w : 0, w, sh) : 0;
    if (b >= 1 || qs == 0) break;
  }
  if (b < 1) return false;
  if (qs) {
    p->grid_defer = num_sms() * b;
    p->wpb_defer = w;
  } else {
    p->grid = num_sms() * b;
  }
  p->wpb = wpb;
  return true;
}

cudaError_t launch_search(const SearchArgs& a, const SearchPlan& p, cudaStream_t s) {
  if (p.fast_qs == 0) return launch_search_general(a, p.wpb, p.grid, s);
  cudaError_t e = launch_search_fast(a, p.fast_qs, p.wpb, p.grid, s);
  if (e != cudaSuccess) return e;
  SearchArgs g = a;
  g.qlist = a.defer;
  g.nq_dev = a.counter + 1;
  return launch_search_general(g, p.wpb_defer, p.grid_defer, s);
}

template <typename T, int DW>
static int bps_t(int warps_per_block, size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(search_kernel<T, DW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, search_kernel<T, DW>, warps_per_block * 32, smem);
  return nb;
}

int search_blocks_per_sm(int dtype, int u8w, int warps_per_block, size_t smem) {
  if (dtype != CNG_F32) return bps_t<__half, 0>(warps_per_block, smem);
  switch (u8w) {
    case 8: return bps_t<float, 8>(warps_per_block, smem);
    case 16: return bps_t<float, 16>(warps_per_block, smem);
    case 24: return bps_t<float, 24>(warps_per_block, smem);
    case 32: return bps_t<float, 32>(warps_per_block, smem);
    default: return bps_t<float, 0>(warps_per_block, smem);
  }
}

// One warp per query: flag[q] = 0 if every coordinate is an integer in [vmin, vmax], else 1;
// with out != null also the 8-bit row out[q][c] = x[q][c] - vmin (0 in the padding).
__global__ void query_check_kernel(const float* __restrict__ Q, int64_t nq, int d, float vmin,
                                   float vmax, int u8w, uint8_t* __restrict__ out,
                                   uint8_t* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = w0; q < nq; q += nw) {
    bool bad = false;
    for (int c = lane; c < d; c += 32) {
      const float x = Q[q * d + c];
      bad |= !(x == rintf(x)) || !(x >= vmin && x <= vmax);
      if (out) out[q * (u8w * 4) + c] = (uint8_t)(int)fminf(fmaxf(x - vmin, 0.f), 255.f);
    }
    if (out)
      for (int c = d + lane; c < u8w * 4; c += 32) out[q * (u8w * 4) + c] = 0;
    const unsigned b = __ballot_sync(FULL, bad);
    if (lane == 0) flag[q] = b ? 1 : 0;
  }
}

cudaError_t launch_query_check(const float* Q, int64_t nq, int d, float vmin, float vmax, int u8w,
                               uint8_t* out, uint8_t* flag, cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nq * 32 + 255) / 256, (int64_t)num_sms() * 8));
  count_launch();
  query_check_kernel<<<grid, 256, 0, s>>>(Q, nq, d, vmin, vmax, u8w, out, flag);
  return cudaGetLastError();
}

}  // namespace cng
