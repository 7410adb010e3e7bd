// k_mlp.cu -- training of the learned early-stop network (not part of the paper's method; the
// paper's search stops only by Alg. 1's rule).
//
// Network: 16 -> 64 -> 64 -> 1, ReLU, logit z; loss = mean binary cross-entropy with logits
//   l(z, y) = max(z, 0) - z y + log(1 + exp(-|z|)).
// Parameters (FP32 master copy), flat: W1[64][16] b1[64] W2[64][64] b2[64] w3[64] b3[1].
// Samples: one per (training query, hop t <= max_trace) of a traced plain search; features as
// in the search kernel, label y = (t >= last hop at which the query's top-k list changed).
// Inputs are standardised with the training set's per-feature mean and standard deviation.
// Optimiser: Adam (beta 0.9 / 0.999, eps 1e-8); minibatch rows drawn with replacement by a
// counter-based hash of (seed, step, slot).  Gradients: each CTA handles 128 samples and writes
// its partial gradient; partials are summed in CTA order, so training is deterministic.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "mlp_internal.h"
#include "search_internal.h"

namespace cng {

constexpr int MT = 128;  // samples (threads) per CTA

CNG_DEV uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// ---- samples from traces ---------------------------------------------------------------------
// counts[q] = min(hops[q], T); offsets by an exclusive scan in one CTA (sequential chunks).
__global__ void trace_offsets_kernel(const int32_t* __restrict__ hops, int64_t nq, int T,
                                     int64_t* __restrict__ off) {
  __shared__ int64_t carry;
  __shared__ int64_t ws[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b = 0; b < nq; b += blockDim.x) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < nq ? min(hops[i], T) : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t w = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(FULL, w, o);
        if (lane >= o) w += t;
      }
      ws[lane] = w;
    }
    __syncthreads();
    int64_t incl = x + (warp > 0 ? ws[warp - 1] : 0) + carry;
    if (i < nq) off[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[nq] = carry;
}

__global__ void flatten_kernel(const float* __restrict__ feats, const int32_t* __restrict__ hops,
                               const int32_t* __restrict__ tlc, const int64_t* __restrict__ off,
                               int64_t nq, int T, float* __restrict__ X, float* __restrict__ y) {
  int64_t q = blockIdx.x;
  if (q >= nq) return;
  const int c = min(hops[q], T);
  const int64_t o = off[q];
  for (int e = threadIdx.x; e < c * 16; e += blockDim.x) {
    int t = e >> 4, j = e & 15;
    X[(o + t) * 16 + j] = feats[((int64_t)q * T + t) * 16 + j];
    if (j == 0) y[o + t] = (t + 1 >= tlc[q]) ? 1.f : 0.f;
  }
}

// per-feature sum and sum of squares in double (one partial per CTA, then one CTA sums them)
__global__ void __launch_bounds__(256) feat_stats_kernel(const float* __restrict__ X, int64_t N,
                                                         double* __restrict__ part) {
  __shared__ double ws[8][32];
  double a[16], b[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = b[j] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      double v = X[i * 16 + j];
      a[j] += v;
      b[j] += v * v;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a[j] += __shfl_xor_sync(FULL, a[j], o);
      b[j] += __shfl_xor_sync(FULL, b[j], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      ws[warp][j] = a[j];
      ws[warp][16 + j] = b[j];
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = 0;
    for (int w = 0; w < 8; ++w) x += ws[w][threadIdx.x];
    part[blockIdx.x * 32 + threadIdx.x] = x;
  }
}

__global__ void feat_norm_kernel(const double* __restrict__ part, int nparts, int64_t N,
                                 float* __restrict__ mu, float* __restrict__ sg) {
  int j = threadIdx.x;
  if (j >= 16) return;
  double x = 0, z = 0;
  for (int p = 0; p < nparts; ++p) {
    x += part[p * 32 + j];
    z += part[p * 32 + 16 + j];
  }
  double m = x / (double)N;
  double v = z / (double)N - m * m;
  mu[j] = (float)m;
  sg[j] = (float)sqrt(v > 1e-12 ? v : 1e-12);
}

__global__ void standardise_kernel(float* __restrict__ X, int64_t N, const float* __restrict__ mu,
                                   const float* __restrict__ sg) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= N * 16) return;
  int j = (int)(e & 15);
  X[e] = (X[e] - mu[j]) / sg[j];
}

// ---- forward + backward --------------------------------------------------------------------------
// One thread per sample; rows = idx ? idx[i] : i.  Writes the CTA's partial gradient and loss.
__global__ void __launch_bounds__(MT)
mlp_fwd_bwd_kernel(const float* __restrict__ P, const float* __restrict__ X, const float* __restrict__ Y,
                   int64_t N, int B, uint64_t seed, int64_t step, float inv_scale,
                   float* __restrict__ part, float* __restrict__ part_loss) {
  extern __shared__ float sm[];
  float* w = sm;                         // MLP_NPARAMS
  float* xs = w + MLP_NPARAMS_PAD;       // [MT][16]
  float* h1 = xs + MT * 16;              // [MT][65] (pad: conflict-free columns)
  float* h2 = h1 + MT * 65;              // [MT][65]
  float* g2 = h2 + MT * 65;              // [MT][65] dL/da2
  float* g1 = g2 + MT * 65;              // [MT][65] dL/da1
  __shared__ float dzs[MT];
  __shared__ float ls[MT];
  const int t = threadIdx.x;
  for (int i = t; i < MLP_NPARAMS; i += MT) w[i] = P[i];
  const float* W1 = w;
  const float* b1 = W1 + 64 * 16;
  const float* W2 = b1 + 64;
  const float* b2 = W2 + 64 * 64;
  const float* w3 = b2 + 64;
  const float* b3 = w3 + 64;
  const int s = blockIdx.x * MT + t;
  const bool live = s < B;
  int64_t row = 0;
  if (live) {
    row = seed ? (int64_t)(splitmix64(seed ^ ((uint64_t)step * 0x100000001B3ull + (uint64_t)s)) %
                           (uint64_t)N)
               : (int64_t)s;
  }
  for (int j = 0; j < 16; ++j) xs[t * 16 + j] = live ? X[row * 16 + j] : 0.f;
  __syncthreads();
  float z = b3[0];
  for (int o = 0; o < 64; ++o) {
    float a = b1[o];
#pragma unroll
    for (int i = 0; i < 16; ++i) a = fmaf(W1[o * 16 + i], xs[t * 16 + i], a);
    h1[t * 65 + o] = fmaxf(a, 0.f);
  }
  for (int o = 0; o < 64; ++o) {
    float a = b2[o];
    for (int i = 0; i < 64; ++i) a = fmaf(W2[o * 64 + i], h1[t * 65 + i], a);
    float r = fmaxf(a, 0.f);
    h2[t * 65 + o] = r;
    z = fmaf(w3[o], r, z);
  }
  const float y = live ? Y[row] : 0.f;
  const float sig = 1.f / (1.f + expf(-z));
  const float dz = live ? (sig - y) * inv_scale : 0.f;
  dzs[t] = dz;
  ls[t] = live ? fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z))) : 0.f;
  for (int o = 0; o < 64; ++o) g2[t * 65 + o] = h2[t * 65 + o] > 0.f ? dz * w3[o] : 0.f;
  for (int i = 0; i < 64; ++i) {
    float a = 0.f;
    for (int o = 0; o < 64; ++o) a = fmaf(W2[o * 64 + i], g2[t * 65 + o], a);
    g1[t * 65 + i] = h1[t * 65 + i] > 0.f ? a : 0.f;
  }
  __syncthreads();
  // parameter gradients of this CTA's samples (fixed summation order over samples)
  float* out = part + (size_t)blockIdx.x * MLP_NPARAMS;
  for (int e = t; e < 64 * 16; e += MT) {  // W1[o][i]
    int o = e >> 4, i = e & 15;
    float a = 0.f;
    for (int q = 0; q < MT; ++q) a = fmaf(g1[q * 65 + o], xs[q * 16 + i], a);
    out[e] = a;
  }
  if (t < 64) {  // b1, b2, w3
    float a = 0.f, c = 0.f, d = 0.f;
    for (int q = 0; q < MT; ++q) {
      a += g1[q * 65 + t];
      c += g2[q * 65 + t];
      d = fmaf(dzs[q], h2[q * 65 + t], d);
    }
    out[64 * 16 + t] = a;
    out[64 * 16 + 64 + 64 * 64 + t] = c;
    out[64 * 16 + 64 + 64 * 64 + 64 + t] = d;
  }
  for (int e = t; e < 64 * 64; e += MT) {  // W2[o][i]
    int o = e >> 6, i = e & 63;
    float a = 0.f;
    for (int q = 0; q < MT; ++q) a = fmaf(g2[q * 65 + o], h1[q * 65 + i], a);
    out[64 * 16 + 64 + e] = a;
  }
  if (t == 0) {
    float a = 0.f, l = 0.f;
    for (int q = 0; q < MT; ++q) {
      a += dzs[q];
      l += ls[q];
    }
    out[MLP_NPARAMS - 1] = a;
    part_loss[blockIdx.x] = l;
  }
}

__global__ void reduce_grad_kernel(const float* __restrict__ part, int nparts,
                                   const float* __restrict__ part_loss, float loss_scale,
                                   float* __restrict__ grad, float* __restrict__ loss) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MLP_NPARAMS) {
    float a = 0.f;
    for (int c = 0; c < nparts; ++c) a += part[(size_t)c * MLP_NPARAMS + p];
    grad[p] = a;
  }
  if (p == 0 && loss) {
    float l = 0.f;
    for (int c = 0; c < nparts; ++c) l += part_loss[c];
    *loss = l * loss_scale;
  }
}

__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t t, float lr) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAMS) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float gi = g[p];
  float mi = b1 * m[p] + (1.f - b1) * gi;
  float vi = b2 * v[p] + (1.f - b2) * gi * gi;
  m[p] = mi;
  v[p] = vi;
  float mh = mi / (1.f - powf(b1, (float)t));
  float vh = vi / (1.f - powf(b2, (float)t));
  P[p] -= lr * mh / (sqrtf(vh) + eps);
}

// Kaiming-uniform weights, zero biases, from the counter-based generator.
__global__ void mlp_init_kernel(float* __restrict__ P, uint64_t seed) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NPARAMS) return;
  float bound = 0.f;
  if (p < 64 * 16) bound = sqrtf(6.f / 16.f);
  else if (p >= 64 * 16 + 64 && p < 64 * 16 + 64 + 64 * 64) bound = sqrtf(6.f / 64.f);
  else if (p >= 64 * 16 + 64 + 64 * 64 + 64 && p < MLP_NPARAMS - 1) bound = sqrtf(6.f / 64.f);
  uint64_t r = splitmix64(seed * 0x9E3779B97F4A7C15ull + (uint64_t)p);
  float u = (float)(r >> 40) * (1.f / 16777216.f);  // [0, 1)
  P[p] = bound * (2.f * u - 1.f);
}

// FP32 master parameters + normalisation -> packed inference block (BF16 weights).
__global__ void pack_model_kernel(const float* __restrict__ P, const float* __restrict__ mu,
                                  const float* __restrict__ sg, unsigned char* __restrict__ blk) {
  // output-major rows padded to 24 and 72 elements (the pads are zero)
  __nv_bfloat16* W1b = reinterpret_cast<__nv_bfloat16*>(blk);
  __nv_bfloat16* W2b = W1b + 64 * 24;
  float* f = reinterpret_cast<float*>(W2b + 64 * 72);
  const float* W1 = P;
  const float* b1 = W1 + 64 * 16;
  const float* W2 = b1 + 64;
  const float* b2 = W2 + 64 * 64;
  const float* w3 = b2 + 64;
  const float* b3 = w3 + 64;
  for (int e = threadIdx.x; e < 64 * 24; e += blockDim.x) {
    const int o = e / 24, i = e % 24;
    W1b[e] = __float2bfloat16_rn(i < 16 ? W1[o * 16 + i] : 0.f);
  }
  for (int e = threadIdx.x; e < 64 * 72; e += blockDim.x) {
    const int o = e / 72, i = e % 72;
    W2b[e] = __float2bfloat16_rn(i < 64 ? W2[o * 64 + i] : 0.f);
  }
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    f[e] = b1[e];
    f[64 + e] = b2[e];
    f[128 + e] = w3[e];
  }
  if (threadIdx.x < 4) f[192 + threadIdx.x] = threadIdx.x == 0 ? b3[0] : 0.f;
  if (threadIdx.x < 16) {
    f[196 + threadIdx.x] = mu[threadIdx.x];
    f[212 + threadIdx.x] = sg[threadIdx.x];
  }
}

// ---- host-side launchers ---------------------------------------------------------------------------
size_t mlp_fwd_bwd_smem() { return (size_t)(MLP_NPARAMS_PAD + MT * 16 + 4 * MT * 65) * sizeof(float); }
int mlp_parts(int B) { return (B + MT - 1) / MT; }

cudaError_t launch_mlp_grad(const float* P, const float* X, const float* Y, int64_t N, int B,
                            uint64_t seed, int64_t step, float* part, float* part_loss, float* grad,
                            float* loss, cudaStream_t s) {
  const size_t sh = mlp_fwd_bwd_smem();
  cudaError_t e = cudaFuncSetAttribute(mlp_fwd_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  if (e != cudaSuccess) return e;
  const int parts = mlp_parts(B);
  count_launch();
  mlp_fwd_bwd_kernel<<<parts, MT, sh, s>>>(P, X, Y, N, B, seed, step, 1.f / (float)B, part, part_loss);
  count_launch();
  reduce_grad_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(part, parts, part_loss, 1.f / (float)B,
                                                               grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* P, float* m, float* v, const float* g, int64_t t, float lr, cudaStream_t s) {
  count_launch();
  adam_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(P, m, v, g, t, lr);
  return cudaGetLastError();
}

cudaError_t launch_mlp_init(float* P, uint64_t seed, cudaStream_t s) {
  count_launch();
  mlp_init_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(P, seed);
  return cudaGetLastError();
}

cudaError_t launch_pack_model(const float* P, const float* mu, const float* sg, void* blk, cudaStream_t s) {
  count_launch();
  pack_model_kernel<<<1, 256, 0, s>>>(P, mu, sg, (unsigned char*)blk);
  return cudaGetLastError();
}

cudaError_t launch_samples(const float* feats, const int32_t* hops, const int32_t* tlc, int64_t nq, int T,
                           int64_t* off, float* X, float* y, cudaStream_t s) {
  count_launch();
  flatten_kernel<<<(unsigned)nq, 128, 0, s>>>(feats, hops, tlc, off, nq, T, X, y);
  return cudaGetLastError();
}

cudaError_t launch_offsets(const int32_t* hops, int64_t nq, int T, int64_t* off, cudaStream_t s) {
  count_launch();
  trace_offsets_kernel<<<1, 1024, 0, s>>>(hops, nq, T, off);
  return cudaGetLastError();
}

cudaError_t launch_standardise(float* X, int64_t N, double* part, float* mu, float* sg, cudaStream_t s) {
  const int nparts = 64;
  count_launch();
  feat_stats_kernel<<<nparts, 256, 0, s>>>(X, N, part);
  count_launch();
  feat_norm_kernel<<<1, 32, 0, s>>>(part, nparts, N, mu, sg);
  count_launch();
  standardise_kernel<<<(unsigned)((N * 16 + 255) / 256), 256, 0, s>>>(X, N, mu, sg);
  return cudaGetLastError();
}

}  // namespace cng
