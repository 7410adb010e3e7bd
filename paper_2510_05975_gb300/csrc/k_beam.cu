// k_beam.cu -- the paper's candidate route (Alg. 3 phase 2, Sec. 4.1): each point's candidate
// list is the C closest points visited by a beam search (Alg. 1) for that point on a K-NN graph
// G0, started from the navigating node.  The search itself runs in the batched search kernels
// with the stored points as queries (k = C + 1, queue Lb >= C + 1: the final queue holds the
// Lb closest visited points, so its first C + 1 entries contain the C closest visited points
// other than p); the kernels here number the queries and drop each point from its own list.
#include "cng_internal.h"
#include "device_common.cuh"
#include "launch_count.h"

namespace cng {

__global__ void iota_kernel(int32_t* a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

// Row p of ids / dists [n][C + 1] (ascending (D, id)) without p itself: the first C others go
// to cand / cdist [n][C].  A row with fewer than C others (a search that visited too few
// points) is reported with ST_BOUNDS.
__global__ void strip_self_kernel(const int32_t* __restrict__ ids, const float* __restrict__ dists,
                                  int64_t n, int C, int32_t* __restrict__ cand, float* __restrict__ cdist,
                                  uint32_t* status) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* ri = ids + p * (C + 1);
    const float* rd = dists + p * (C + 1);
    int c = 0;
    for (int t = 0; t <= C && c < C; ++t) {
      const int32_t v = ri[t];
      if (v < 0 || v == (int32_t)p) continue;
      cand[p * C + c] = v;
      cdist[p * C + c] = rd[t];
      ++c;
    }
    if (c < C) {
      atomicOr(status, ST_BOUNDS);
      for (; c < C; ++c) {
        cand[p * C + c] = -1;
        cdist[p * C + c] = INFINITY;
      }
    }
  }
}

// G0 rows given by the caller: every entry must be a point id other than the row's own, or -1
// padding after the last neighbour.
__global__ void check_knn_graph_kernel(const int32_t* __restrict__ g, int64_t n, int K, uint32_t* status) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * K; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / K;
    const int j = (int)(e - p * K);
    const int32_t v = g[e];
    const bool pad_ok = v >= 0 || j + 1 == K || g[e + 1] < 0;
    if (v >= n || v < -1 || v == (int32_t)p || !pad_ok) atomicOr(status, ST_BOUNDS);
  }
}

static int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

cudaError_t launch_iota(int32_t* a, int64_t n, cudaStream_t s) {
  count_launch();
  iota_kernel<<<grid_for(n), 256, 0, s>>>(a, n);
  return cudaGetLastError();
}

cudaError_t launch_strip_self(const int32_t* ids, const float* dists, int64_t n, int C, int32_t* cand,
                              float* cdist, uint32_t* status, cudaStream_t s) {
  count_launch();
  strip_self_kernel<<<grid_for(n), 256, 0, s>>>(ids, dists, n, C, cand, cdist, status);
  return cudaGetLastError();
}

cudaError_t launch_check_knn_graph(const int32_t* g, int64_t n, int K, uint32_t* status, cudaStream_t s) {
  count_launch();
  check_knn_graph_kernel<<<grid_for(n * K), 256, 0, s>>>(g, n, K, status);
  return cudaGetLastError();
}

}  // namespace cng
