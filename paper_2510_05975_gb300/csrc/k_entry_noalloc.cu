// k_entry_noalloc.cu -- the navigating node without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this result: processes
// whose device memory belongs to another allocator (a framework's caching pool that must see
// every byte, or a fixed arena budgeted at start-up), and latency-bound loops that cannot wait
// for the allocator's implicit synchronisation.  For them
// cng_entry_noalloc computes the same navigating node as cng_build -- the point nearest the
// centroid, ties to the smaller id, the centroid summed in blocks of 4,096 rows in FP64; for
// CNG_L2 and CNG_IP_AS_L2 builds (a CNG_IP build takes its entry on augmented rows) --
// using only the caller's input and output plus a file-scope device array.
//
// The array holds the block partial sums, the centroid and the two argmin words.  It has a
// fixed size (ENTRY_SCRATCH_DOUBLES doubles, 4 MiB) and exists on every GPU that loads this
// library until the process exits.  Its device address is looked up once per device with
// cudaGetSymbolAddress (host code must not use the array's name as a device pointer) during
// the first call on that device, so that first call should be made before any stream capture.
// Every call uses the same array: the argmin words are re-initialised by the kernels of each
// call, the partial sums are fully rewritten; calls that overlap on the GPU race with each
// other.
#include <mutex>

#include "cng_internal.h"
#include "device_common.cuh"
#include "launch_count.h"

namespace cng {

constexpr int64_t ENTRY_SCRATCH_DOUBLES = 1 << 19;  // 4 MiB
constexpr int ENTRY_BLOCK = 4096;                   // rows per centroid block sum

static __device__ __align__(256) double g_entry_scratch[ENTRY_SCRATCH_DOUBLES];

template <typename T>
__global__ void na_centroid_part(const T* __restrict__ X, int64_t n, int d,
                                 double* __restrict__ part) {
  int j = blockIdx.y * blockDim.x + threadIdx.x;
  if (j >= d) return;
  int64_t b0 = (int64_t)blockIdx.x * ENTRY_BLOCK;
  int64_t e = min(n, b0 + ENTRY_BLOCK);
  double s = 0.0;
  for (int64_t i = b0; i < e; ++i) s = __dadd_rn(s, (double)to_f(X[i * d + j]));
  part[(int64_t)blockIdx.x * d + j] = s;
}

__global__ void na_centroid_final(const double* __restrict__ part, int nblk, int64_t n, int d,
                                  double* __restrict__ cen, unsigned long long* best) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j == 0) {
    best[0] = ~0ull;
    best[1] = ~0ull;
  }
  if (j >= d) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) t = __dadd_rn(t, part[(int64_t)b * d + j]);
  cen[j] = __ddiv_rn(t, (double)n);
}

template <typename T>
CNG_DEV unsigned long long na_dist_bits(const T* __restrict__ x, const double* cs, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) {
    double t = __dsub_rn(cs[j], (double)to_f(x[j]));
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return (unsigned long long)__double_as_longlong(__dsqrt_rn(s));
}

// pass 1: smallest canonical distance (as bits; distances are >= 0); pass 2: smallest id at it
template <typename T, bool PICK>
__global__ void __launch_bounds__(256) na_entry_pass(const T* __restrict__ X, int64_t n, int d,
                                                     const double* __restrict__ cen,
                                                     unsigned long long* best) {
  extern __shared__ double cs[];
  for (int j = threadIdx.x; j < d; j += blockDim.x) cs[j] = cen[j];
  __syncthreads();
  const unsigned long long target = PICK ? best[0] : 0ull;
  unsigned long long mine = ~0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long b = na_dist_bits(X + i * d, cs, d);
    if (PICK) {
      if (b == target) mine = min(mine, (unsigned long long)i);
    } else {
      mine = min(mine, b);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_xor_sync(FULL, mine, o));
  if ((threadIdx.x & 31) == 0 && mine != ~0ull) atomicMin(&best[PICK ? 1 : 0], mine);
}

__global__ void na_entry_write(const unsigned long long* best, int32_t* out) {
  *out = (int32_t)best[1];
}

static std::mutex g_mu;
static double* g_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_entry_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

int64_t entry_noalloc_need(int64_t n, int d) {
  const int64_t nblk = (n + ENTRY_BLOCK - 1) / ENTRY_BLOCK;
  return nblk * d + d + 2;
}

int64_t entry_noalloc_capacity() { return ENTRY_SCRATCH_DOUBLES; }

template <typename T>
static cudaError_t run(const T* X, int64_t n, int d, int32_t* out, cudaStream_t s, double* base) {
  const int nblk = (int)((n + ENTRY_BLOCK - 1) / ENTRY_BLOCK);
  double* part = base;
  double* cen = part + (int64_t)nblk * d;
  unsigned long long* best = reinterpret_cast<unsigned long long*>(cen + d);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
  count_launch();
  na_centroid_part<T><<<dim3(nblk, (d + 127) / 128), 128, 0, s>>>(X, n, d, part);
  count_launch();
  na_centroid_final<<<(d + 127) / 128, 128, 0, s>>>(part, nblk, n, d, cen, best);
  count_launch();
  na_entry_pass<T, false><<<grid, 256, d * sizeof(double), s>>>(X, n, d, cen, best);
  count_launch();
  na_entry_pass<T, true><<<grid, 256, d * sizeof(double), s>>>(X, n, d, cen, best);
  count_launch();
  na_entry_write<<<1, 1, 0, s>>>(best, out);
  return cudaGetLastError();
}

cudaError_t launch_entry_noalloc(const void* X, int dtype, int64_t n, int d, int32_t* out,
                                 cudaStream_t s) {
  double* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return e;
  return dtype == CNG_F32 ? run((const float*)X, n, d, out, s, base)
                          : run((const __half*)X, n, d, out, s, base);
}

}  // namespace cng

namespace cng {
cng_status fail(cng_status st, const std::string& msg);
}

extern "C" cng_status cng_entry_noalloc(const void* points, int32_t dtype, int64_t n, int32_t d,
                                        int32_t* entry, void* stream) {
  using namespace cng;
  if (!points || !entry) return fail(CNG_E_INVAL, "points and entry must be non-NULL");
  if (dtype != CNG_F32 && dtype != CNG_F16) return fail(CNG_E_INVAL, "dtype must be CNG_F32 or CNG_F16");
  if (n < 1 || n > 0x7fffffffLL || d < 1 || d > 4096)
    return fail(CNG_E_INVAL, "need 1 <= n < 2^31 and 1 <= d <= 4096");
  const int64_t need = entry_noalloc_need(n, d);
  if (need > entry_noalloc_capacity())
    return fail(CNG_E_INVAL, "cng_entry_noalloc: ceil(n / 4096) * d + d + 2 = " + std::to_string(need) +
                                 " doubles exceeds the fixed scratch of " +
                                 std::to_string(entry_noalloc_capacity()) + " doubles (4 MiB)");
  for (const void* p : {points, (const void*)entry}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return fail(CNG_E_INVAL, "points and entry must be device memory");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return fail(CNG_E_INVAL, "points and entry must be device memory");
  }
  cudaError_t e = launch_entry_noalloc(points, dtype, n, d, entry, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(CNG_E_CUDA, std::string("cng_entry_noalloc: ") + cudaGetErrorString(e));
  return CNG_OK;
}
