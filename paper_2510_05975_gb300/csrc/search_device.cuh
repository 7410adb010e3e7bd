// search_device.cuh -- device helpers shared by the two batched search kernels (Alg. 1):
// the visited filter, the stop network's inference, exact 8-bit distances and a warp sort.
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"

namespace cng {

constexpr int SQ_ROWSLOTS = 3;  // 32-lane slices of an adjacency row (row stride R + 8 <= 96)

CNG_DEV uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Visited filter (open addressing, <= 8 probes).  Returns 0 if v is known to be visited, 1 if
// it was not and is now recorded, 2 if its probe slots are all taken by other points: then v
// may or may not have been seen (slots never empty, so a recorded point is always found before
// a free slot, and a point once refused is refused again).
CNG_DEV int visit3(int32_t* H, int hmask, int32_t v) {
  const uint32_t h = hash32((uint32_t)v) & hmask;
  for (int p = 0; p < 8; ++p) {  // one compare-and-swap per probe: claims a free slot or reads it
    const int32_t old = atomicCAS(H + ((h + p) & hmask), -1, v);
    if (old == -1) return 1;
    if (old == v) return 0;
  }
  return 2;
}

// True unless v is known to be visited.
CNG_DEV bool visit(int32_t* H, int hmask, int32_t v) { return visit3(H, hmask, v) != 0; }

CNG_DEV float lgf(float x) { return logf(fmaxf(x, 1e-30f)); }

// The stop model in shared memory: BF16 weights (inputs-major, so lane o reads W[i][o]
// conflict-free), FP32 biases and input normalisation.
struct StopSmem {
  const __nv_bfloat16* W1T;  // [16][64]
  const __nv_bfloat16* W2T;  // [64][64]
  const float *b1, *b2, *w3, *b3, *mu, *sg;
};
CNG_DEV StopSmem stop_smem(const unsigned char* mb) {
  StopSmem m;
  m.W1T = reinterpret_cast<const __nv_bfloat16*>(mb);
  m.W2T = m.W1T + 16 * 64;
  const float* f = reinterpret_cast<const float*>(m.W2T + 64 * 64);
  m.b1 = f;
  m.b2 = f + 64;
  m.w3 = f + 128;
  m.b3 = f + 192;
  m.mu = f + 196;
  m.sg = f + 212;
  return m;
}

// Logit of the 16-64-64-1 ReLU network for the features held by lanes 0..15 (FP32 math on
// BF16 weights); every lane returns the same value.
CNG_DEV float mlp_logit(const StopSmem& m, float f, int lane) {
  const float xh = lane < 16 ? (f - m.mu[lane]) / m.sg[lane] : 0.f;
  float a0 = m.b1[lane], a1 = m.b1[lane + 32];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float xi = __shfl_sync(FULL, xh, i);
    a0 = fmaf(__bfloat162float(m.W1T[i * 64 + lane]), xi, a0);
    a1 = fmaf(__bfloat162float(m.W1T[i * 64 + lane + 32]), xi, a1);
  }
  const float h0 = fmaxf(a0, 0.f), h1 = fmaxf(a1, 0.f);
  float c0 = m.b2[lane], c1 = m.b2[lane + 32];
#pragma unroll 8
  for (int i = 0; i < 32; ++i) {
    const float hi = __shfl_sync(FULL, h0, i);
    c0 = fmaf(__bfloat162float(m.W2T[i * 64 + lane]), hi, c0);
    c1 = fmaf(__bfloat162float(m.W2T[i * 64 + lane + 32]), hi, c1);
  }
#pragma unroll 8
  for (int i = 0; i < 32; ++i) {
    const float hi = __shfl_sync(FULL, h1, i);
    c0 = fmaf(__bfloat162float(m.W2T[(i + 32) * 64 + lane]), hi, c0);
    c1 = fmaf(__bfloat162float(m.W2T[(i + 32) * 64 + lane + 32]), hi, c1);
  }
  float z = m.w3[lane] * fmaxf(c0, 0.f) + m.w3[lane + 32] * fmaxf(c1, 0.f);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(FULL, z, o);
  return z + m.b3[0];
}

// One lane's exact squared distance to 8-bit row v: the whole row in DW / 4 independent 16-byte
// loads, then |q|^2 + |v|^2 - 2 <q, v> in integers (below 2^24 for d <= 128).
template <int DW>
CNG_DEV uint32_t u8_lane_d2(const uint4* qu, uint32_t qn, const uint8_t* __restrict__ U, int64_t v) {
  const uint4* r = reinterpret_cast<const uint4*>(U + v * (DW * 4));
  uint4 x[DW / 4];
#pragma unroll
  for (int q = 0; q < DW / 4; ++q) x[q] = __ldg(r + q);
  uint32_t dot = 0, nv = 0;
#pragma unroll
  for (int q = 0; q < DW / 4; ++q) {
    const uint4 y = qu[q];
    dot = __dp4a(x[q].x, y.x, dot); dot = __dp4a(x[q].y, y.y, dot);
    dot = __dp4a(x[q].z, y.z, dot); dot = __dp4a(x[q].w, y.w, dot);
    nv = __dp4a(x[q].x, x[q].x, nv); nv = __dp4a(x[q].y, x[q].y, nv);
    nv = __dp4a(x[q].z, x[q].z, nv); nv = __dp4a(x[q].w, x[q].w, nv);
  }
  return qn + nv - 2u * dot;
}

template <int DW>
CNG_DEV float u8_lane_sqdist(const uint4* qu, uint32_t qn, const uint8_t* __restrict__ U, int64_t v) {
  return (float)u8_lane_d2<DW>(qu, qn, U, v);
}

// Ascending bitonic sort of one key per lane across the warp (lane i ends with the i-th
// smallest).
template <typename K>
CNG_DEV K warp_sort32(K key, int lane) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const K o = __shfl_xor_sync(FULL, key, j);
      const bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
      key = take_min ? (o < key ? o : key) : (o > key ? o : key);
    }
  return key;
}

}  // namespace cng
