// k_mips.cu -- maximum inner product search as L2 search on augmented vectors, sm_103a.
//
// The paper's graph is built over a metric space (Sec. 2.1).  Inner-product ranking of rows of
// any norm becomes Euclidean ranking after appending one coordinate: with M^2 = max_i |x_i|^2,
//   x' = [x, sqrt(M^2 - |x|^2)],  q' = [q, 0]   =>   |q' - x'|^2 = |q|^2 + M^2 - 2 <q, x>,
// so the L2-nearest augmented rows are the rows of largest <q, x>.  Every |x|^2 is summed in
// FP64 over the coordinates in order (each square is exact), M^2 is their maximum, and the
// extra coordinate is the correctly rounded FP64 square root rounded once to FP32.
#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "mips_internal.h"

namespace cng {
namespace {

template <typename T>
__global__ void mips_norm_kernel(const T* __restrict__ X, int64_t n, int d, double* __restrict__ nrm2,
                                 unsigned long long* __restrict__ max_bits) {
  double local_max = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    const T* x = X + i * d;
    for (int j = 0; j < d; ++j) {
      const double v = (double)to_f(x[j]);
      s = __dadd_rn(s, __dmul_rn(v, v));
    }
    nrm2[i] = s;
    local_max = fmax(local_max, s);
  }
  // non-negative doubles order like their bit patterns
  atomicMax(max_bits, (unsigned long long)__double_as_longlong(local_max));
}

template <typename T>
__global__ void mips_augment_kernel(const T* __restrict__ X, int64_t n, int d,
                                    const double* __restrict__ nrm2,
                                    const unsigned long long* __restrict__ max_bits,
                                    float* __restrict__ out) {
  const double M2 = __longlong_as_double((long long)*max_bits);
  const int dd = d + 1;
  const int64_t total = n * dd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / dd;
    const int j = (int)(e - i * dd);
    out[e] = j < d ? to_f(X[i * d + j]) : __double2float_rn(sqrt(__dadd_rn(M2, -nrm2[i])));
  }
}

__global__ void append_zero_kernel(const float* __restrict__ Q, int64_t nq, int d,
                                   float* __restrict__ out) {
  const int dd = d + 1;
  const int64_t total = nq * dd;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / dd;
    const int j = (int)(e - i * dd);
    out[e] = j < d ? Q[i * d + j] : 0.f;
  }
}

int grid_for(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)num_sms() * 16));
}

}  // namespace

cudaError_t launch_mips_augment(const void* X, int dtype, int64_t n, int d, double* nrm2,
                                unsigned long long* max_bits, float* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  count_launch();
  if (dtype == CNG_F32)
    mips_norm_kernel<float><<<grid_for(n), 256, 0, s>>>((const float*)X, n, d, nrm2, max_bits);
  else
    mips_norm_kernel<__half><<<grid_for(n), 256, 0, s>>>((const __half*)X, n, d, nrm2, max_bits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  count_launch();
  if (dtype == CNG_F32)
    mips_augment_kernel<float><<<grid_for(n * (d + 1)), 256, 0, s>>>((const float*)X, n, d, nrm2,
                                                                      max_bits, out);
  else
    mips_augment_kernel<__half><<<grid_for(n * (d + 1)), 256, 0, s>>>((const __half*)X, n, d, nrm2,
                                                                       max_bits, out);
  return cudaGetLastError();
}

cudaError_t launch_append_zero(const float* Q, int64_t nq, int d, float* out, cudaStream_t s) {
  count_launch();
  append_zero_kernel<<<grid_for(nq * (d + 1)), 256, 0, s>>>(Q, nq, d, out);
  return cudaGetLastError();
}

}  // namespace cng
