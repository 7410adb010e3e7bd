// device_common.cuh -- device helpers shared by the alpha-CNG kernels (sm_103a).
//
// Numerics contract (the paper fixes none; Sec. 2.1 only asks for a metric):
//  * canonical distance: D(x,y) = sqrt(sum_i (x_i - y_i)^2) in IEEE double, index order,
//    one rounding per operation (explicit __d*_rn intrinsics, so no contraction);
//  * fast distance: FP32 direct differences, 4 interleaved accumulators per lane and a
//    G-lane shuffle tree; relative error of the squared distance <= (chain + 3) * 2^-24 with
//    chain <= 4 * ceil(dpad / (16 G)) + 2 + log2 G (<= 40 for every supported shape);
//  * an FP32 decision between a and b is trusted when |a - b| > band * max(|a|, |b|) with
//    band >= 5e-6 > 2 * that bound; otherwise it is re-decided with the canonical distance.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "status_bits.h"

#define CNG_DEV __device__ __forceinline__

namespace cng {

constexpr unsigned FULL = 0xffffffffu;


CNG_DEV void set_status(uint32_t* st, uint32_t bits) { atomicOr(st, bits); }

CNG_DEV float to_f(float v) { return v; }
CNG_DEV float to_f(__half v) { return __half2float(v); }

// ---- canonical FP64 distance --------------------------------------------------------------
template <typename TA, typename TB>
CNG_DEV double canon_sqdist(const TA* x, const TB* y, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) {
    double t = __dsub_rn((double)to_f(x[i]), (double)to_f(y[i]));
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}
// FP32 rows: the same operations in the same order, with 16-byte loads when both rows are
// 16-byte aligned (so the loads run ahead of the sequential FP64 sum).
CNG_DEV double canon_sqdist(const float* x, const float* y, int d) {
  double s = 0.0;
  int i = 0;
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0) {
#pragma unroll 4
    for (; i + 4 <= d; i += 4) {
      const float4 a = *reinterpret_cast<const float4*>(x + i);
      const float4 b = *reinterpret_cast<const float4*>(y + i);
      const double t0 = __dsub_rn((double)a.x, (double)b.x), t1 = __dsub_rn((double)a.y, (double)b.y);
      const double t2 = __dsub_rn((double)a.z, (double)b.z), t3 = __dsub_rn((double)a.w, (double)b.w);
      s = __dadd_rn(s, __dmul_rn(t0, t0));
      s = __dadd_rn(s, __dmul_rn(t1, t1));
      s = __dadd_rn(s, __dmul_rn(t2, t2));
      s = __dadd_rn(s, __dmul_rn(t3, t3));
    }
  }
  for (; i < d; ++i) {
    const double t = __dsub_rn((double)x[i], (double)y[i]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

template <typename TA, typename TB>
CNG_DEV double canon_dist(const TA* x, const TB* y, int d) {
  return __dsqrt_rn(canon_sqdist(x, y, d));
}

// Def. 2 / Eq. 1 in double: prunes iff Dpu > alpha * Duv + t, t = (alpha + 1) * tau.
CNG_DEV bool rule64(double Dpu, double Duv, double alpha, double t) {
  double rhs = __dadd_rn(__dmul_rn(alpha, Duv), t);
  return Dpu > rhs;
}

CNG_DEV bool near_tie(float a, float b, float band) {
  return fabsf(a - b) <= band * fmaxf(fabsf(a), fabsf(b));
}

// Order-preserving map float -> uint32 (total order on non-NaN floats).
CNG_DEV uint32_t fkey(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
CNG_DEV float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// (distance, id) packed so that unsigned comparison is the lexicographic (d, id) order.
CNG_DEV uint64_t pack_key(float d, int32_t id) {
  return ((uint64_t)fkey(d) << 32) | (uint32_t)id;
}
CNG_DEV float key_dist(uint64_t k) { return fkey_inv((uint32_t)(k >> 32)); }
CNG_DEV int32_t key_id(uint64_t k) { return (int32_t)(uint32_t)(k & 0xffffffffu); }

// ---- FP32 distances by a group of G lanes ------------------------------------------------
// Vectors are stored padded to dpad elements (a multiple of 32 for float, of 64 for half);
// lane g of the group reads 16-byte chunks g, g + G, g + 2G, ...
CNG_DEV void acc4(float4 a, float4 b, float& s) {
  float t;
  t = a.x - b.x; s = fmaf(t, t, s);
  t = a.y - b.y; s = fmaf(t, t, s);
  t = a.z - b.z; s = fmaf(t, t, s);
  t = a.w - b.w; s = fmaf(t, t, s);
}
CNG_DEV float4 h8lo(uint4 v) {
  float2 a = __half22float2(*reinterpret_cast<__half2*>(&v.x));
  float2 b = __half22float2(*reinterpret_cast<__half2*>(&v.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
CNG_DEV float4 h8hi(uint4 v) {
  float2 a = __half22float2(*reinterpret_cast<__half2*>(&v.z));
  float2 b = __half22float2(*reinterpret_cast<__half2*>(&v.w));
  return make_float4(a.x, a.y, b.x, b.y);
}

template <int G>
CNG_DEV float group_reduce(float s) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  return s;
}

// q: float vector (shared or global), y: stored row (float), partial sum for this lane.
template <int G>
CNG_DEV float part_sqdist(const float* __restrict__ q, const float* __restrict__ y, int dpad, int g) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  int nch = dpad >> 2;
  int c = g;
  for (; c + 3 * G < nch; c += 4 * G) {
    float4 a0 = q4[c], a1 = q4[c + G], a2 = q4[c + 2 * G], a3 = q4[c + 3 * G];
    float4 b0 = __ldg(y4 + c), b1 = __ldg(y4 + c + G), b2 = __ldg(y4 + c + 2 * G), b3 = __ldg(y4 + c + 3 * G);
    acc4(a0, b0, s0); acc4(a1, b1, s1); acc4(a2, b2, s2); acc4(a3, b3, s3);
  }
  for (; c < nch; c += G) acc4(q4[c], __ldg(y4 + c), s0);
  return (s0 + s1) + (s2 + s3);
}
template <int G>
CNG_DEV float part_sqdist(const float* __restrict__ q, const __half* __restrict__ y, int dpad, int g) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const uint4* y8 = reinterpret_cast<const uint4*>(y);
  int nch = dpad >> 3;  // 8 halves per 16-byte chunk
  int c = g;
  for (; c + G < nch; c += 2 * G) {
    uint4 b0 = __ldg(y8 + c), b1 = __ldg(y8 + c + G);
    acc4(q4[2 * c], h8lo(b0), s0); acc4(q4[2 * c + 1], h8hi(b0), s1);
    acc4(q4[2 * (c + G)], h8lo(b1), s2); acc4(q4[2 * (c + G) + 1], h8hi(b1), s3);
  }
  for (; c < nch; c += G) {
    uint4 b0 = __ldg(y8 + c);
    acc4(q4[2 * c], h8lo(b0), s0); acc4(q4[2 * c + 1], h8hi(b0), s1);
  }
  return (s0 + s1) + (s2 + s3);
}

// Load a stored row into a float buffer (shared), all lanes of the calling group/warp.
CNG_DEV void load_row(float* dst, const float* __restrict__ src, int dpad, int t, int nt) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int c = t; c < (dpad >> 2); c += nt) d4[c] = __ldg(s4 + c);
}
CNG_DEV void load_row(float* dst, const __half* __restrict__ src, int dpad, int t, int nt) {
  const uint4* s8 = reinterpret_cast<const uint4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int c = t; c < (dpad >> 3); c += nt) {
    uint4 v = __ldg(s8 + c);
    d4[2 * c] = h8lo(v);
    d4[2 * c + 1] = h8hi(v);
  }
}

// ---- warp-cooperative selection for the fused top-L' row buffers -----------------------
// A row buffer holds `cnt` packed (score key, id) entries.  warp_compact keeps the Lp
// smallest keys (ties at the cut broken arbitrarily but deterministically by buffer order),
// moves them to the front and returns the key of the largest kept entry.  All 32 lanes call
// it with the same arguments.  CAP_PER_LANE bounds cnt <= 32 * CAP_PER_LANE.
template <int CAP_PER_LANE>
CNG_DEV uint32_t warp_compact(uint64_t* buf, int cnt, int Lp, int lane) {
  uint32_t k[CAP_PER_LANE];
  uint64_t e[CAP_PER_LANE];
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) {
    int idx = i * 32 + lane;
    e[i] = idx < cnt ? buf[idx] : ~0ull;
    k[i] = (uint32_t)(e[i] >> 32);
  }
  __syncwarp();
  // radix select (MSB first) of the Lp-th smallest key (1-based rank)
  uint32_t prefix = 0, mask = 0;
  int need = Lp;
  for (int b = 31; b >= 0; --b) {
    uint32_t bit = 1u << b;
    int c0 = 0;
#pragma unroll
    for (int i = 0; i < CAP_PER_LANE; ++i) {
      bool m = (i * 32 + lane < cnt) && ((k[i] & mask) == prefix) && !(k[i] & bit);
      c0 += __popc(__ballot_sync(FULL, m));
    }
    if (c0 < need) { need -= c0; prefix |= bit; }
    mask |= bit;
  }
  const uint32_t kth = prefix;  // `need` entries equal to kth are kept
  int out = 0, eq_taken = 0;
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) {
    bool valid = i * 32 + lane < cnt;
    bool lt = valid && k[i] < kth;
    bool eq = valid && k[i] == kth;
    unsigned beq = __ballot_sync(FULL, eq);
    int eq_rank = eq_taken + __popc(beq & ((1u << lane) - 1));
    bool keep = lt || (eq && eq_rank < need);
    eq_taken += __popc(beq);
    unsigned bk = __ballot_sync(FULL, keep);
    if (keep) buf[out + __popc(bk & ((1u << lane) - 1))] = e[i];
    out += __popc(bk);
  }
  __syncwarp();
  return kth;
}

}  // namespace cng
