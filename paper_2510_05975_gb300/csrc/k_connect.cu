// k_connect.cu -- Alg. 3 phase 4 (connectivity) on the GPU.
//
// The paper adds "necessary edges" from the DFS tree of the navigating node s to every point
// outside it, in line with NSG.  Reading used here, in rounds until every point is reachable:
//   reached = points reachable from s (frontier BFS);
//   for every unreached p: r(p) = the first result of beam-search(G, x_p, s, Lc, Lc) on the
//     current graph whose row has a free slot at the start of the round (the batched search
//     kernel with point ids as queries);
//   if some unreached p without any in-edge has an r(p): each such p gets the edge r(p) -> p,
//     a row taking its points in ascending order while it has free slots (one claim-and-link
//     step per slot; such a p can be reached in no other way);
//   otherwise every r named by some r(p) gets the edge r -> (smallest such p).
// Rows have stride R + slots so that phase-3 rows keep all of their edges.
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

__global__ void has_in_kernel(const int32_t* __restrict__ adj, const int32_t* __restrict__ deg, int Rs,
                              int64_t n, int32_t* __restrict__ has_in) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * Rs) return;
  const int64_t u = e / Rs;
  const int j = (int)(e - u * Rs);
  if (j < deg[u]) has_in[adj[e]] = 1;
}

// r(p) with the degrees at the start of the round (before any edge of the round is added)
__global__ void pick_kernel(const int32_t* __restrict__ U, const int32_t* __restrict__ r, int nu,
                            int kc, const int32_t* __restrict__ deg, int Rs,
                            const int32_t* __restrict__ has_in, int32_t* __restrict__ rp,
                            int* __restrict__ nz) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  int32_t pick = -1;
  for (int t = 0; t < kc; ++t) {
    const int32_t c = r[(int64_t)i * kc + t];
    if (c >= 0 && deg[c] < Rs) {
      pick = c;
      break;
    }
  }
  rp[i] = pick;
  if (pick >= 0 && !has_in[U[i]]) atomicAdd(nz, 1);
}

__global__ void claim_kernel(const int32_t* __restrict__ U, const int32_t* __restrict__ rp, int nu,
                             const int32_t* __restrict__ has_in, int zonly,
                             const int32_t* __restrict__ deg, int Rs, int32_t* __restrict__ best) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  const int32_t r = rp[i];
  if (r < 0 || deg[r] >= Rs) return;
  const int32_t p = U[i];
  if (zonly && has_in[p]) return;
  atomicMin(&best[r], p);
}

// The claim of row r is decided (the previous launch finished): its winner alone writes row r.
__global__ void link_kernel(const int32_t* __restrict__ U, int32_t* __restrict__ rp, int nu,
                            int32_t* __restrict__ best, int32_t* __restrict__ adj,
                            int32_t* __restrict__ deg, int Rs, int* __restrict__ added) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  const int32_t r = rp[i];
  if (r < 0) return;
  const int32_t p = U[i];
  if (best[r] != p) return;
  const int dg = deg[r];  // < Rs: claim_kernel checked it
  adj[(int64_t)r * Rs + dg] = p;
  deg[r] = dg + 1;
  best[r] = 0x7fffffff;
  rp[i] = -1;
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

cudaError_t launch_has_in(const int32_t* adj, const int32_t* deg, int Rs, int64_t n, int32_t* has_in,
                          cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(has_in, 0, (size_t)n * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  count_launch();
  has_in_kernel<<<blocks(n * Rs), 256, 0, st>>>(adj, deg, Rs, n, has_in);
  return cudaGetLastError();
}

cudaError_t launch_pick(const int32_t* U, const int32_t* r, int nu, int kc, const int32_t* deg,
                        int Rs, const int32_t* has_in, int32_t* rp, int* nz_dev, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(nz_dev, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  count_launch();
  pick_kernel<<<blocks(nu), 256, 0, st>>>(U, r, nu, kc, deg, Rs, has_in, rp, nz_dev);
  return cudaGetLastError();
}

cudaError_t launch_claim_link(const int32_t* U, int32_t* rp, int nu, const int32_t* has_in, int zonly,
                              int32_t* best, int32_t* adj, int32_t* deg, int Rs, int* added_dev,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(added_dev, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  count_launch();
  claim_kernel<<<blocks(nu), 256, 0, st>>>(U, rp, nu, has_in, zonly, deg, Rs, best);
  count_launch();
  link_kernel<<<blocks(nu), 256, 0, st>>>(U, rp, nu, best, adj, deg, Rs, added_dev);
  return cudaGetLastError();
}

cudaError_t launch_fill(int32_t* a, int64_t n, int32_t v, cudaStream_t st) {
  count_launch();
  fill_kernel<<<blocks(n), 256, 0, st>>>(a, n, v);
  return cudaGetLastError();
}

}  // namespace cng
