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

// Stop feature `lane` (0..15) after hop `hops`, in the order of the stop model's feature list,
// from the search state: D0 entry distance, D1 / Dk / DL distances of Q's first, min(k, |Q|)-th
// and last entries, Du the hop vertex's distance, hist[h & 63] = Dk after hop h, tlc the last
// hop that changed the top-k ids, U unexplored entries, ins this hop's points left in Q.  Every
// lane takes one logarithm of its own argument (no lane-dependent branches around logf).
CNG_DEV float stop_feature(int lane, float D0, float D1, float Dk, float DL, float Du,
                           const float* hist, int hops, int tlc, int U, int len, int ins, int L,
                           int R) {
  const float lD0 = lgf(D0), lDk = lgf(Dk);
  const int h = lane >= 6 && lane < 12 ? max(hops - (1 << (lane - 6)), 0) : 0;
  const float hv = hist[h & 63];
  float A = D0, B = 0.f;  // f = lg(A) - B
  if (lane == 1) A = 1.f + (float)hops;
  else if (lane == 2) { A = D1; B = lD0; }
  else if (lane == 3) { A = Dk; B = lD0; }
  else if (lane == 4) { A = DL; B = lD0; }
  else if (lane == 5) { A = Du; B = lDk; }
  else if (lane >= 6 && lane < 12) { A = hv; B = lDk; }
  else if (lane == 12) A = 1.f + (float)(hops - tlc);
  const float lg = lgf(A) - B;
  if (lane == 13) return (float)U / (float)L;
  if (lane == 14) return (float)len / (float)L;
  if (lane == 15) return (float)ins / (float)R;
  return lg;
}

// The stop model in shared memory: BF16 weights stored output-major with padded rows (W1
// [64][24], W2 [64][72] elements; the pads keep a warp's fragment loads free of bank
// conflicts), then FP32 biases, w3 and the input normalisation.
constexpr int STOP_W1_LD = 24, STOP_W2_LD = 72;
struct StopSmem {
  const uint32_t* W1;  // bf16 pairs, row stride STOP_W1_LD / 2 words
  const uint32_t* W2;  // bf16 pairs, row stride STOP_W2_LD / 2 words
  const float *b1, *b2, *w3, *b3, *mu, *sg;
};
CNG_DEV StopSmem stop_smem(const unsigned char* mb) {
  StopSmem m;
  m.W1 = reinterpret_cast<const uint32_t*>(mb);
  m.W2 = m.W1 + 64 * STOP_W1_LD / 2;
  const float* f = reinterpret_cast<const float*>(m.W2 + 64 * STOP_W2_LD / 2);
  m.b1 = f;
  m.b2 = f + 64;
  m.w3 = f + 128;
  m.b3 = f + 192;
  m.mu = f + 196;
  m.sg = f + 212;
  return m;
}

// Two FP32 values as one BF16 pair (lower half = lo) and the BF16 pair of their residuals, so
// that hi + lo carries about 16 significant bits of each value.
CNG_DEV void split_bf16x2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// D = A B + D on the tensor cores (m16n8k16, BF16 operands, FP32 accumulators).
CNG_DEV void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                      uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Logit of the 16-64-64-1 ReLU network for the features held by lanes 0..15; every lane
// returns the same value.  The single input row is row 0 of m16n8k16 MMAs (lanes 0..3 hold
// it; the other rows are zero): layer 1 is 8 n-tiles of one k-step, layer 2 is 8 n-tiles of 4
// k-steps, and each activation enters as a BF16 pair hi + lo (two MMAs), so the products are
// those of the BF16 weights with ~16-bit activations, accumulated in FP32.  Layer 1's output
// tiles 2 kk and 2 kk + 1 are, lane for lane, the A fragment of layer 2's k-step kk.
static __device__ __noinline__ float mlp_logit(const StopSmem& m, float f, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const bool row0 = lane < 4;
  const float xh = lane < 16 ? (f - m.mu[lane]) / m.sg[lane] : 0.f;
  const float x0 = __shfl_sync(FULL, xh, 2 * t), x1 = __shfl_sync(FULL, xh, 2 * t + 1);
  const float x8 = __shfl_sync(FULL, xh, 2 * t + 8), x9 = __shfl_sync(FULL, xh, 2 * t + 9);
  uint32_t ah0, al0, ah2, al2;
  split_bf16x2(x0, x1, ah0, al0);
  split_bf16x2(x8, x9, ah2, al2);
  if (!row0) ah0 = al0 = ah2 = al2 = 0u;
  // layer 1 -> A fragments of layer 2 (hi and lo parts of k-steps 0..3)
  uint32_t h2hi[4][2], h2lo[4][2];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t* w = m.W1 + (8 * j + g) * (STOP_W1_LD / 2) + t;
    const float2 bias = *reinterpret_cast<const float2*>(m.b1 + 8 * j + 2 * t);
    float d[4] = {bias.x, bias.y, 0.f, 0.f};
    mma_bf16(d, ah0, 0u, ah2, 0u, w[0], w[4]);
    mma_bf16(d, al0, 0u, al2, 0u, w[0], w[4]);
    uint32_t hi, lo;
    split_bf16x2(fmaxf(d[0], 0.f), fmaxf(d[1], 0.f), hi, lo);
    h2hi[j >> 1][j & 1] = row0 ? hi : 0u;
    h2lo[j >> 1][j & 1] = row0 ? lo : 0u;
  }
  // layer 2 and the output layer
  float z = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 bias = *reinterpret_cast<const float2*>(m.b2 + 8 * j + 2 * t);
    float d[4] = {bias.x, bias.y, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint32_t* w = m.W2 + (8 * j + g) * (STOP_W2_LD / 2) + 8 * kk + t;
      mma_bf16(d, h2hi[kk][0], 0u, h2hi[kk][1], 0u, w[0], w[4]);
      mma_bf16(d, h2lo[kk][0], 0u, h2lo[kk][1], 0u, w[0], w[4]);
    }
    const float2 w3 = *reinterpret_cast<const float2*>(m.w3 + 8 * j + 2 * t);
    z = fmaf(w3.x, fmaxf(d[0], 0.f), z);
    z = fmaf(w3.y, fmaxf(d[1], 0.f), z);
  }
  z = row0 ? z : 0.f;
  z += __shfl_xor_sync(FULL, z, 1);
  z += __shfl_xor_sync(FULL, z, 2);
  return __shfl_sync(FULL, z, 0) + m.b3[0];
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
