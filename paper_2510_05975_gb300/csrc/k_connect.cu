// k_connect.cu -- Alg. 3 phase 4 (connectivity) on the GPU.
//
// The paper adds "necessary edges" from the DFS tree of the navigating node s to every point
// outside it, in line with NSG.  Reading used here, in rounds until every point is reachable:
//   reached = points reachable from s (frontier BFS);
//   for every unreached p: r(p) = the nearest result of beam-search(G, x_p, s, Lc, 1) on the
//     current graph (the batched search kernel with point ids as queries);
//   every reached r named by some r(p) gets the edge r -> (smallest such p) if its row has a
//   free slot; rows have stride R + 8 so that phase-3 rows keep all of their edges.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"

namespace cng {

__global__ void bfs_init_kernel(int32_t* __restrict__ reached, int64_t n, int32_t s,
                                int32_t* __restrict__ frontier, int* __restrict__ counts) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) reached[i] = (i == s);
  if (i == 0) {
    frontier[0] = s;
    counts[0] = 1;  // frontier size
    counts[1] = 0;  // next size
    counts[2] = 0;  // unreached
    counts[3] = 0;  // edges added
  }
}

__global__ void bfs_expand_kernel(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg,
                                  int Rs, const int32_t* __restrict__ frontier, int nf,
                                  int32_t* __restrict__ reached, int32_t* __restrict__ next,
                                  int* __restrict__ ncount) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nf * Rs) return;
  int i = (int)(e / Rs), j = (int)(e - (int64_t)i * Rs);
  int32_t u = frontier[i];
  if (j >= deg[u]) return;
  int32_t v = adj[(int64_t)u * Rs + j];
  if (atomicExch(&reached[v], 1) == 0) next[atomicAdd(ncount, 1)] = v;
}

__global__ void collect_unreached_kernel(const int32_t* __restrict__ reached, int64_t n,
                                         int32_t* __restrict__ U, int* __restrict__ nu) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !reached[i]) U[atomicAdd(nu, 1)] = (int32_t)i;
}

// deg is read before add_edges_kernel changes it: the snapshot of the round's start.
__global__ void pick_kernel(const int32_t* __restrict__ U, const int32_t* __restrict__ r, int nu,
                            int kc, const int32_t* __restrict__ deg, int Rs,
                            int32_t* __restrict__ best) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  for (int t = 0; t < kc; ++t) {
    int32_t c = r[(int64_t)i * kc + t];
    if (c >= 0 && deg[c] < Rs) {
      atomicMin(&best[c], U[i]);
      return;
    }
  }
}

__global__ void add_edges_kernel(int32_t* __restrict__ best, int64_t n, int32_t* __restrict__ adj,
                                 int32_t* __restrict__ deg, int Rs, int* __restrict__ added) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  int32_t p = best[r];
  if (p == 0x7fffffff) return;
  best[r] = 0x7fffffff;
  int dg = deg[r];  // < Rs: pick_kernel only names rows with a free slot
  adj[r * Rs + dg] = p;
  deg[r] = dg + 1;
  atomicAdd(added, 1);
}

__global__ void fill_kernel(int32_t* __restrict__ a, int64_t n, int32_t v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

static int blocks(int64_t n) { return (int)((n + 255) / 256); }

cudaError_t launch_bfs(const int32_t* adj, const int32_t* deg, int Rs, int64_t n, int32_t s,
                       int32_t* reached, int32_t* fa, int32_t* fb, int* counts_dev,
                       int* counts_host, cudaStream_t st) {
  count_launch();
  bfs_init_kernel<<<blocks(n), 256, 0, st>>>(reached, n, s, fa, counts_dev);
  int nf = 1;
  while (nf > 0) {
    cudaMemsetAsync(counts_dev + 1, 0, sizeof(int), st);
    count_launch();
    bfs_expand_kernel<<<blocks((int64_t)nf * Rs), 256, 0, st>>>(adj, deg, Rs, fa, nf, reached, fb,
                                                               counts_dev + 1);
    cudaError_t e = cudaMemcpyAsync(counts_host + 1, counts_dev + 1, sizeof(int),
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    nf = counts_host[1];
    std::swap(fa, fb);
  }
  return cudaGetLastError();
}

cudaError_t launch_collect(const int32_t* reached, int64_t n, int32_t* U, int* nu_dev, cudaStream_t st) {
  cudaMemsetAsync(nu_dev, 0, sizeof(int), st);
  count_launch();
  collect_unreached_kernel<<<blocks(n), 256, 0, st>>>(reached, n, U, nu_dev);
  return cudaGetLastError();
}

cudaError_t launch_pick_add(const int32_t* U, const int32_t* r, int nu, int kc, int32_t* best,
                            int64_t n, int32_t* adj, int32_t* deg, int Rs, int* added_dev,
                            cudaStream_t st) {
  cudaMemsetAsync(added_dev, 0, sizeof(int), st);
  count_launch();
  pick_kernel<<<blocks(nu), 256, 0, st>>>(U, r, nu, kc, deg, Rs, best);
  count_launch();
  add_edges_kernel<<<blocks(n), 256, 0, st>>>(best, n, adj, deg, Rs, added_dev);
  return cudaGetLastError();
}

cudaError_t launch_fill(int32_t* a, int64_t n, int32_t v, cudaStream_t st) {
  count_launch();
  fill_kernel<<<blocks(n), 256, 0, st>>>(a, n, v);
  return cudaGetLastError();
}

}  // namespace cng
