// api.cu -- C ABI of libcng.so (declared in include/cng.h): argument checks, device memory,
// phase ordering and statistics of the alpha-CNG build (Alg. 3 phases 1-3, exact candidates)
// and the batched beam search (Alg. 1).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "launch_count.h"
#include "cng_internal.h"
#include "search_internal.h"
#include "mlp_internal.h"
#include "order_internal.h"
#include "screen_tc.h"
#include "mips_internal.h"

namespace cng {

static thread_local std::string g_err = "no error";

std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}

cng_status fail(cng_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? CNG_E_NOMEM : CNG_E_CUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)

// Owns device allocations made during one call; frees them on scope exit.
struct DevPool {
  std::vector<void*> ptrs;
  ~DevPool() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
  void release(void* p) {  // keep p alive beyond the pool
    ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end());
  }
};

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace cng

using namespace cng;

struct cng_index {
  int64_t n = 0;
  int d = 0, dpad = 0, dtype = 0, R = 0, L = 0;
  int metric = CNG_L2;      // CNG_IP: rows (and queries) are augmented by one coordinate
  double mips_M2 = 0.0;     // CNG_IP: the largest squared row norm
  int rs = 0;               // adjacency row stride (R + repair slots)
  int32_t entry = -1;
  int exact = 0;
  float band = 1e-5f;
  void* xs = nullptr;       // stored points [n][dpad]
  int32_t* adj = nullptr;   // [n][R]
  int32_t* deg = nullptr;   // [n]
  int32_t* cand = nullptr;  // [n][L] (keep_lists)
  float* cdist = nullptr;
  int32_t* fwd = nullptr;   // [n][R] (keep_lists)
  int32_t* fdeg = nullptr;
  float vmin = 0.f, vmax = 0.f;  // data value range (exact integer data)
  uint8_t* u8 = nullptr;         // 8-bit rows x - vmin [n][4 u8w] (integer data spanning <= 255)
  int u8w = 0;
  uint8_t* qbuf = nullptr;       // per-search query flags + 8-bit query rows (grown on demand)
  size_t qbuf_cap = 0;
  // search scratch
  int* counter = nullptr;        // SEARCH_COUNTER_INTS
  int32_t* defer = nullptr;      // queries left to the general search kernel (grown on demand)
  int64_t defer_cap = 0;
  char* stage = nullptr;         // device staging of host queries and results (grown on demand)
  size_t stage_cap = 0;
  unsigned long long* tot = nullptr;
  uint32_t* status = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for CUDA-graph capture
  // Calls that use the scratch above are ordered on the GPU: each records `done` on its stream
  // and the next call, if on another stream, waits for it first.
  cudaEvent_t done = nullptr;
  cudaStream_t last_stream = nullptr;
  bool has_last = false;
  std::mutex mu;
  struct GraphEntry {
    SearchArgs args;
    SearchPlan plan;
    cudaStream_t stream;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
};

// Autotuned search launch shapes, shared by every index of the same shape in the process.
struct TunedShape {
  int dev, dtype, dpad, rs, u8w, L, mode;  // key
  int wpb, hash;                      // warps per block, visited-filter slots
};
static std::mutex g_tune_mu;
static std::vector<TunedShape> g_tuned;

struct cng_stop_model {
  float* P = nullptr;     // FP32 master parameters
  float* mu = nullptr;    // [16]
  float* sg = nullptr;    // [16]
  void* blk = nullptr;    // packed inference block (BF16 weights)
};

extern "C" const char* cng_last_error(void) { return g_err.c_str(); }

extern "C" void cng_stop_free(cng_stop_model* m) {
  if (!m) return;
  cudaFree(m->P);
  cudaFree(m->mu);
  cudaFree(m->sg);
  cudaFree(m->blk);
  delete m;
}

// Search scratch (staging areas, deferred-query lists) of freed indexes, kept for the next
// index on the same device so its first host-buffer search allocates nothing.  Bounded: at most
// kScratchKeep buffers; a buffer beyond that is freed.
namespace {
struct ScratchBuf {
  int dev;
  void* p;
  size_t bytes;
};
constexpr size_t kScratchKeep = 8;
std::mutex g_scratch_mu;
std::vector<ScratchBuf> g_scratch;
}  // namespace

static void scratch_give(void* p, size_t bytes) {
  if (!p) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch.size() >= kScratchKeep) {
    cudaFree(p);
    return;
  }
  g_scratch.push_back({dev, p, bytes});
}

// The smallest cached buffer of at least `bytes` on the current device, or a new allocation.
static cudaError_t scratch_take(size_t bytes, void** p, size_t* got) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    int best = -1;
    for (int i = 0; i < (int)g_scratch.size(); ++i)
      if (g_scratch[i].dev == dev && g_scratch[i].bytes >= bytes &&
          (best < 0 || g_scratch[i].bytes < g_scratch[best].bytes))
        best = i;
    if (best >= 0) {
      *p = g_scratch[best].p;
      *got = g_scratch[best].bytes;
      g_scratch.erase(g_scratch.begin() + best);
      return cudaSuccess;
    }
  }
  *got = bytes;
  return cudaMalloc(p, bytes);
}

extern "C" void cng_free(cng_index* ix) {
  if (!ix) return;
  // the scratch goes back to the cache: the index's last call must be complete
  if (ix->has_last) cudaEventSynchronize(ix->done);
  scratch_give(ix->stage, ix->stage_cap);
  scratch_give(ix->defer, (size_t)ix->defer_cap * sizeof(int32_t));
  ix->stage = nullptr;
  ix->defer = nullptr;
  for (auto& g : ix->graphs) cudaGraphExecDestroy(g.exec);
  cudaFree(ix->xs);
  cudaFree(ix->adj);
  cudaFree(ix->deg);
  cudaFree(ix->cand);
  cudaFree(ix->cdist);
  cudaFree(ix->fwd);
  cudaFree(ix->fdeg);
  cudaFree(ix->u8);
  cudaFree(ix->qbuf);
  cudaFree(ix->counter);
  cudaFree(ix->defer);
  cudaFree(ix->stage);
  cudaFree(ix->tot);
  cudaFree(ix->status);
  if (ix->cap_stream) cudaStreamDestroy(ix->cap_stream);
  if (ix->done) cudaEventDestroy(ix->done);
  delete ix;
}

namespace cng {

struct Timer {
  cudaEvent_t ev[8];
  int n = 0;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    for (auto& e : ev) cudaEventCreate(&e);
  }
  ~Timer() {
    for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark() { cudaEventRecord(ev[n++], s); }
  double ms(int a, int b) {
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
};

// Exact candidate lists for m rows against n stored columns (K1 screen -> K2 rerank ->
// rescan).  xr / xc are stored matrices [.][dpad] of `dtype`.  Writes ids [m][L], dist [m][L].
struct KnnInputs {
  const void* xr;
  const void* xc;
  int64_t m, n;
  int d, dpad, dtype;
  int self_excl;
  int L, Lp;
  int screen;   // cng_screen
  float band;
  int exact;
  // tensor-core operands (screen == CNG_SCREEN_TC)
  const void* tc_rows;  // [m][kpad] bf16 / fp16
  const void* tc_cols;  // [n][kpad]
  int kpad;
  int tc_fp16;          // operands are FP16 (else BF16)
  const float* nb_rows;  // ||x_b||^2 of rows
  const float* nb_cols;  // ||y_b||^2 of columns
  const float* rb_rows;
  float rbmax, normmax;
  float scale2;  // operands are scale * x, scores in units of scale^2
  // locality order of the tensor-core operands (tc_rows / tc_cols / nb_cols hold positions)
  const int32_t* perm;
  int wave_start;
  int variant = -1;  // tensor-core screen pipeline variant (-1: autotuned)
  const uint8_t* u8 = nullptr;  // 8-bit rows of the points (rows = columns), or null
  int u8w = 0;
};

static cng_status run_knn(const KnnInputs& in, int32_t* out_ids, float* out_dist, Counters* ctr,
                          double* ms_screen, double* ms_rerank, cudaStream_t s,
                          TcShape* shape = nullptr) {
  DevPool pool;
  int32_t* sids;
  uint32_t* sthr;
  CK(pool.alloc(&sids, (size_t)in.m * in.Lp));
  CK(pool.alloc(&sthr, (size_t)in.m));
  Timer tm(s);
  tm.mark();
  ScreenModel sm{};
  if (in.screen == CNG_SCREEN_TC) {
    TcScreenArgs ta{};
    ta.A = in.tc_rows;
    ta.B = in.tc_cols;
    ta.m = in.m;
    ta.n = in.n;
    ta.kpad = in.kpad;
    ta.fp16 = in.tc_fp16;
    ta.nb = in.nb_cols;
    ta.Lp = in.Lp;
    ta.self_excl = in.self_excl;
    ta.ids = sids;
    ta.thr = sthr;
    ta.status = &ctr->status;
    ta.rowbuf_words = screen_tc_rowbuf_words(in.m, in.n, in.Lp);
    ta.perm = in.perm;
    ta.wave_start = in.wave_start;
    ta.variant = in.variant;
    CK(pool.alloc(&ta.rowbuf, ta.rowbuf_words));
    std::string msg;
    if (in.variant < 0) {  // a first use of this shape times the variants (outside the timing)
      cudaError_t te = launch_screen_tc_tune(ta, s, &msg, &ta.variant);
      if (te != cudaSuccess) return fail(CNG_E_CUDA, "tensor-core screen: " + msg + cudaGetErrorString(te));
      tm.mark();  // the screen's time starts after the tuning trials
    }
    cudaError_t e = launch_screen_tc(ta, s, &msg, shape);
    if (e != cudaSuccess) return fail(CNG_E_CUDA, "tensor-core screen: " + msg + cudaGetErrorString(e));
    sm.kind = 1;
    sm.nb = in.nb_rows;
    sm.rb = in.rb_rows;
    sm.rbmax = in.rbmax;
    sm.normmax = in.normmax;
    sm.acc_err = (float)(in.kpad + 8) * 1.1920929e-7f;  // K terms, 2^-23 per add
    sm.scale2 = in.scale2;
  } else {
    int cpl = 0;
    for (int c : {8, 12, 16, 20})
      if (c * 32 >= in.Lp + 128 + 32) { cpl = c; break; }
    if (!cpl) return fail(CNG_E_UNSUPPORTED, "screened list too long");
    int grid = std::min<int64_t>((in.m + 127) / 128, (int64_t)num_sms() * 2);
    uint64_t* rowbuf;
    CK(pool.alloc(&rowbuf, (size_t)grid * 128 * cpl * 32));
    CK(launch_knn_simt(in.xr, in.m, in.xc, in.n, in.dtype, in.dpad, in.Lp, in.self_excl, rowbuf,
                       cpl, grid, sids, sthr, &ctr->status, s));
    sm.kind = 0;
    sm.rel_err = (float)(in.dpad + 8) * 5.9604645e-8f;
  }
  sm.exact = in.exact;
  tm.mark();
  int32_t* fail_rows;
  float* fail_bound;
  CK(pool.alloc(&fail_rows, (size_t)in.m));
  CK(pool.alloc(&fail_bound, (size_t)in.m));
  CK(launch_rerank(in.xr, in.xc, in.dtype, in.m, in.d, in.dpad, sids, sthr, in.Lp, in.L, sm,
                   in.band, in.exact, out_ids, out_dist, fail_rows, fail_bound, ctr, in.u8, in.u8w,
                   s));
  CK(launch_rescan(in.xr, in.xc, in.dtype, in.m, in.n, in.d, in.dpad, in.self_excl, in.L,
                   fail_rows, fail_bound, ctr, out_ids, out_dist, s));
  tm.mark();
  CK(cudaStreamSynchronize(s));
  const int m0 = tm.n - 3;  // marks: [tuning start,] screen start, screen end, rerank end
  if (ms_screen) *ms_screen = tm.ms(m0, m0 + 1);
  if (ms_rerank) *ms_rerank = tm.ms(m0 + 1, m0 + 2);
  return CNG_OK;
}

static cng_status check_status(uint32_t st) {
  if (st & ST_TIMEOUT) return fail(CNG_E_TIMEOUT, "a bounded device wait ran out");
  if (st & ST_OVERFLOW)
    return fail(CNG_E_UNSUPPORTED, "a candidate row buffer overflowed");
  if (st & ST_CERT) return fail(CNG_E_UNSUPPORTED, "more than 4096 points tie at a candidate boundary");
  if (st & ST_OVF_MERGE) return fail(CNG_E_INTERNAL, "a merged candidate set exceeded its buffer");
  if (st & ST_OVF_RUN)
    return fail(CNG_E_UNSUPPORTED, "more than 256 consecutive near-tied distances (degenerate input)");
  if (st & ST_BOUNDS) return fail(CNG_E_INTERNAL, "device index check failed");
  if (st & ST_SCREEN) return fail(CNG_E_INTERNAL, "screened scores violate the exactness assumption");
  return CNG_OK;
}

// Stored copy + exactness of one point matrix.
struct Prepared {
  void* xs = nullptr;
  void* tc = nullptr;
  float* nb = nullptr;
  float* rb = nullptr;
  PrepStats st{};
};

// Tensor-core operand scale: 1 for integer data with |x| <= 2048 (exact in FP16) and for FP16
// input; otherwise the power of two that puts max |s x| in (4096, 8192], which keeps the FP16
// operands clear of overflow and of the subnormal range (relative rounding 2^-11).
static cng_status operand_scale(const void* const* pts, const int64_t* ns, int count, int dtype,
                                int d, float* scale, cudaStream_t s) {
  *scale = 1.f;
  if (dtype != CNG_F32) return CNG_OK;
  DevPool pool;
  uint32_t* dev;
  CK(pool.alloc(&dev, 2));
  CK(cudaMemsetAsync(dev, 0, 2 * sizeof(uint32_t), s));
  for (int i = 0; i < count; ++i)
    if (ns[i] > 0) CK(launch_absmax(pts[i], dtype, ns[i], d, dev, s));
  uint32_t host[2];
  CK(cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float amax;
  memcpy(&amax, &host[0], 4);
  if (!host[1] && amax <= 2048.f) return CNG_OK;
  if (!(amax > 0.f) || !std::isfinite(amax)) return CNG_OK;
  const int e = (int)std::ceil(std::log2((double)amax));
  *scale = (float)std::ldexp(1.0, 13 - e);
  return CNG_OK;
}

// fp16ops: tensor-core operands in FP16 (scaled by `scale`); else BF16 (unscaled).
static cng_status prepare(DevPool& pool, const void* pts_dev, int dtype, int64_t n, int d,
                          int dpad, int screen, int kpad, Prepared* out, cudaStream_t s,
                          int fp16ops = 1, float scale = 1.f) {
  size_t el = dtype == CNG_F32 ? 4 : 2;
  CK(pool.alloc(reinterpret_cast<char**>(&out->xs), (size_t)n * dpad * el));
  __nv_bfloat16* xb_bf = nullptr;
  __half* xb_h = nullptr;
  if (screen == CNG_SCREEN_TC) {
    if (dtype == CNG_F32 && !fp16ops) {
      CK(pool.alloc(&xb_bf, (size_t)n * kpad));
      out->tc = xb_bf;
    } else {
      CK(pool.alloc(&xb_h, (size_t)n * kpad));
      out->tc = xb_h;
    }
    CK(pool.alloc(&out->nb, (size_t)n + 256));
    CK(pool.alloc(&out->rb, (size_t)n));
    CK(cudaMemsetAsync(out->nb, 0, ((size_t)n + 256) * sizeof(float), s));
  }
  PrepStats* dst;
  CK(pool.alloc(&dst, 1));
  PrepStats init{};
  init.vmin_key = 0xffffffffu;
  CK(cudaMemcpyAsync(dst, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  CK(launch_prep(pts_dev, dtype, n, d, dpad, out->xs, xb_bf, xb_h, kpad, out->nb, out->rb,
                 dtype == CNG_F32 ? scale : 1.f, dst, s));
  CK(cudaMemcpyAsync(&out->st, dst, sizeof(PrepStats), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return CNG_OK;
}

// Self k-NN through the tensor-core screen in a locality order: replaces pr's screening copy by
// one in k-d order and points ki at it (rows and columns are positions, ki->perm the ids).
static cng_status apply_order(DevPool& pool, Prepared* pr, int dtype, int64_t n, int d, int dpad,
                              int kpad, KnnInputs* ki, double* ms, cudaStream_t s) {
  if (order_levels(n) == 0) return CNG_OK;
  Timer to(s);
  to.mark();
  int32_t* perm;
  void* oscr;
  void* xbp;
  float* nbp;
  CK(pool.alloc(&perm, (size_t)n));
  CK(pool.alloc(reinterpret_cast<char**>(&oscr), order_scratch_bytes(n)));
  CK(launch_order(pr->xs, dtype, n, d, dpad, perm, oscr, s));
  CK(pool.alloc(reinterpret_cast<char**>(&xbp), (size_t)n * kpad * 2));
  CK(pool.alloc(&nbp, (size_t)n + 256));
  CK(cudaMemsetAsync(nbp, 0, ((size_t)n + 256) * sizeof(float), s));
  CK(launch_order_gather(pr->tc, pr->nb, perm, n, kpad, xbp, nbp, s));
  to.mark();
  CK(cudaStreamSynchronize(s));
  cudaFree(oscr);
  pool.release(oscr);
  cudaFree(pr->tc);
  pool.release(pr->tc);
  pr->tc = xbp;
  ki->tc_rows = xbp;
  ki->tc_cols = xbp;
  ki->nb_cols = nbp;
  ki->perm = perm;
  ki->wave_start = 1;
  *ms = to.ms(0, 1);
  return CNG_OK;
}

static float key_to_float(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  float f;
  memcpy(&f, &b, 4);
  return f;
}
static float bits_to_float(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}

// 8-bit rows u = x - min(x) hold the data exactly when every coordinate is an integer and the
// span is at most 255; squared distances are then exact 32-bit integers below 2^24.
static bool u8_rows_ok(const PrepStats& st, int d) {
  if (st.nonint) return false;
  const double lo = key_to_float(st.vmin_key), hi = key_to_float(st.vmax_key);
  const double span = hi - lo;
  return span >= 0.0 && span <= 255.0 && (double)d * span * span < 16777216.0 && u8_words(d) > 0;
}

// Squared distances are exact FP32 integers when every coordinate is an integer and
// d * span^2 < 2^24 (span = max - min coordinate); the tensor-core screen additionally needs
// |coordinate| <= 256 (exact in bf16) and ||x||^2 < 2^24.
static int exact_int(const PrepStats& st, int d, int screen, int bf16ops = 0) {
  if (st.nonint) return 0;
  double lo = key_to_float(st.vmin_key), hi = key_to_float(st.vmax_key);
  double span = hi - lo;
  if ((double)d * span * span >= 16777216.0) return 0;
  if (screen == CNG_SCREEN_TC) {
    // integers are exact up to 2048 in FP16, up to 256 in BF16
    if (std::max(std::fabs(lo), std::fabs(hi)) > (bf16ops ? 256.0 : 2048.0)) return 0;
    double nm = bits_to_float(st.normmax_bits);
    if (nm * nm >= 8388608.0) return 0;
  }
  return 1;
}

}  // namespace cng

static cng_status validate_build(const void* points, int32_t dtype, int64_t n, int32_t d,
                                 const cng_build_params* p) {
  if (!points || !p) return fail(CNG_E_INVAL, "points and params must be non-NULL");
  if (dtype != CNG_F32 && dtype != CNG_F16) return fail(CNG_E_INVAL, "dtype must be CNG_F32 or CNG_F16");
  if (n < 2 || n > 0x7fffffffLL) return fail(CNG_E_INVAL, "n must be in [2, 2^31 - 1]");
  if (d < 1 || d > 4096) return fail(CNG_E_INVAL, "d must be in [1, 4096]");
  if (p->metric == CNG_IP && d > 4095) return fail(CNG_E_INVAL, "CNG_IP needs d <= 4095");
  if (p->L < 1 || p->L > 256 || p->L >= n) return fail(CNG_E_INVAL, "L must satisfy 1 <= L <= 256 and L < n");
  if (p->R < 1 || p->R > p->L || p->R > 64) return fail(CNG_E_INVAL, "R must satisfy 1 <= R <= min(L, 64)");
  if (!(p->alpha > 0.0) || !std::isfinite(p->alpha)) return fail(CNG_E_INVAL, "alpha must be a positive finite number");
  if (!(p->tau >= 0.0) || !std::isfinite(p->tau)) return fail(CNG_E_INVAL, "tau must be finite and >= 0");
  if (p->metric != CNG_L2 && p->metric != CNG_IP_AS_L2 && p->metric != CNG_IP)
    return fail(CNG_E_INVAL, "unknown metric");
  if (p->screen != CNG_SCREEN_FP32 && p->screen != CNG_SCREEN_TC && p->screen != CNG_SCREEN_TC_BF16)
    return fail(CNG_E_INVAL, "unknown screen");
  if (!(p->tie_band >= 5e-6) || p->tie_band > 0.01) return fail(CNG_E_INVAL, "tie_band must be in [5e-6, 0.01]");
  if (p->margin < 0 || p->margin > 256) return fail(CNG_E_INVAL, "margin must be in [0, 256]");
  if (p->connect_L > 256) return fail(CNG_E_INVAL, "connect_L must be <= 256");
  if (p->adaptive) {
    if (!(p->alpha0 > 0.0) || !std::isfinite(p->alpha0) || !std::isfinite(p->alpha_max) ||
        !(p->alpha_max >= p->alpha0) || !(p->dalpha > 0.0) ||
        (p->alpha_max - p->alpha0) / p->dalpha > 1000.0)
      return fail(CNG_E_INVAL,
                  "adaptive pruning needs 0 < alpha0 <= alpha_max, dalpha > 0 and at most 1001 steps");
  }
  if (p->repair_slots < 0 || p->repair_slots > 64) return fail(CNG_E_INVAL, "repair_slots must be in [0, 64]");
  if (p->screen_variant < 0 || p->screen_variant > screen_tc_variants())
    return fail(CNG_E_INVAL, "screen_variant must be in [0, " + std::to_string(screen_tc_variants()) + "]");
  if (p->candidates != CNG_CAND_EXACT && p->candidates != CNG_CAND_BEAM)
    return fail(CNG_E_INVAL, "unknown candidates route");
  if (p->candidates == CNG_CAND_BEAM) {
    const int K = p->knn_K > 0 ? p->knn_K : 200, Lb = p->beam_L > 0 ? p->beam_L : p->L + 1;
    if (p->L > 255) return fail(CNG_E_INVAL, "CNG_CAND_BEAM needs L <= 255");
    if (K < p->L || K > 256 || K >= n) return fail(CNG_E_INVAL, "CNG_CAND_BEAM needs L <= knn_K <= 256 and knn_K < n");
    if (Lb < p->L + 1 || Lb > 256) return fail(CNG_E_INVAL, "CNG_CAND_BEAM needs L + 1 <= beam_L <= 256");
    if (p->metric == CNG_IP && p->knn_graph)
      return fail(CNG_E_INVAL, "CNG_IP builds its own G0 (knn_graph must be NULL)");
    if (p->knn_graph && !is_device_ptr(p->knn_graph)) return fail(CNG_E_INVAL, "knn_graph must be device memory");
  }
  return CNG_OK;
}

extern "C" cng_status cng_build(const void* points, int32_t dtype, int64_t n, int32_t d,
                                const cng_build_params* params, void* stream, cng_index** out,
                                cng_build_stats* stats) {
  if (!out) return fail(CNG_E_INVAL, "out must be non-NULL");
  *out = nullptr;
  cng_status vs = validate_build(points, dtype, n, d, params);
  if (vs != CNG_OK) return vs;
  cudaStream_t s = (cudaStream_t)stream;
  const cng_build_params& P = *params;
  if (P.metric == CNG_IP) {
    // maximum inner product: the L2 index of the augmented rows [x, sqrt(M^2 - |x|^2)]
    DevPool apool;
    const size_t el = dtype == CNG_F32 ? 4 : 2;
    const void* src = points;
    if (!is_device_ptr(points)) {
      char* tmp;
      CK(apool.alloc(&tmp, (size_t)n * d * el));
      CK(cudaMemcpyAsync(tmp, points, (size_t)n * d * el, cudaMemcpyHostToDevice, s));
      src = tmp;
    }
    double* nrm2;
    unsigned long long* mbits;
    float* aug;
    CK(apool.alloc(&nrm2, (size_t)n));
    CK(apool.alloc(&mbits, 1));
    CK(apool.alloc(&aug, (size_t)n * (d + 1)));
    CK(launch_mips_augment(src, dtype, n, d, nrm2, mbits, aug, s));
    unsigned long long hb = 0;
    CK(cudaMemcpyAsync(&hb, mbits, sizeof(hb), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cng_build_params q = P;
    q.metric = CNG_L2;
    cng_status st = cng_build(aug, CNG_F32, n, d + 1, &q, stream, out, stats);
    if (st == CNG_OK) {
      (*out)->metric = CNG_IP;
      memcpy(&(*out)->mips_M2, &hb, sizeof(double));
    }
    return st;
  }
  // BF16 operands (unscaled) for f32 data on request; FP16 input is screened in FP16 as stored
  const int bf16ops = P.screen == CNG_SCREEN_TC_BF16 && dtype == CNG_F32;
  int screen = P.screen == CNG_SCREEN_TC_BF16 ? CNG_SCREEN_TC : P.screen;
  if (screen == CNG_SCREEN_TC && !tc_screen_supported(d, dtype == CNG_F16)) screen = CNG_SCREEN_FP32;
  DevPool pool;
  Timer tm(s);
  tm.mark();  // 0
  const size_t el = dtype == CNG_F32 ? 4 : 2;
  const void* pts = points;
  if (!is_device_ptr(points)) {
    void* tmp;
    CK(pool.alloc(reinterpret_cast<char**>(&tmp), (size_t)n * d * el));
    CK(cudaMemcpyAsync(tmp, points, (size_t)n * d * el, cudaMemcpyHostToDevice, s));
    pts = tmp;
  }
  const int dpad = round_up(d, dtype == CNG_F32 ? 32 : 64);
  const int kpad = round_up(d, 64);
  Prepared pr;
  float scale = 1.f;
  if (screen == CNG_SCREEN_TC && !bf16ops) {
    const void* pl[1] = {pts};
    const int64_t nl[1] = {n};
    cng_status ss = operand_scale(pl, nl, 1, dtype, d, &scale, s);
    if (ss != CNG_OK) return ss;
  }
  cng_status st = prepare(pool, pts, dtype, n, d, dpad, screen, kpad, &pr, s, !bf16ops, scale);
  if (st != CNG_OK) return st;
  if (P.metric == CNG_IP_AS_L2 && bits_to_float(pr.st.unitdev_bits) > 1e-3f)
    return fail(CNG_E_INVAL, "CNG_IP_AS_L2 requires unit-norm rows (| ||x|| - 1 | <= 1e-3)");
  const int exact = exact_int(pr.st, d, screen, bf16ops);
  const float band = (float)P.tie_band;
  tm.mark();  // 1
  // phase 1: navigating node
  int nblk = (int)((n + 4095) / 4096);
  double *part, *cen;
  unsigned long long* best;
  int32_t* d_entry;
  CK(pool.alloc(&part, (size_t)nblk * d + (size_t)n));
  CK(pool.alloc(&cen, (size_t)d));
  CK(pool.alloc(&best, 2));
  CK(pool.alloc(&d_entry, 1));
  CK(launch_entry(pr.xs, dtype, n, d, dpad, part, cen, best, d_entry, s));
  tm.mark();  // 2
  // phase 2a: exact candidate lists
  Counters* ctr;
  CK(pool.alloc(&ctr, 1));
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
  const int L = P.L, R = P.R;
  const int Lp = (int)std::min<int64_t>((int64_t)L + P.margin, n - 1);
  int32_t* cand;
  float* cdist;
  CK(pool.alloc(&cand, (size_t)n * L));
  CK(pool.alloc(&cdist, (size_t)n * L));
  KnnInputs ki{};
  ki.xr = pr.xs;
  ki.xc = pr.xs;
  ki.m = n;
  ki.n = n;
  ki.d = d;
  ki.dpad = dpad;
  ki.dtype = dtype;
  ki.self_excl = 1;
  ki.L = L;
  ki.Lp = Lp;
  ki.screen = screen;
  ki.band = band;
  ki.exact = exact;
  ki.tc_rows = pr.tc;
  ki.tc_cols = pr.tc;
  ki.kpad = kpad;
  ki.tc_fp16 = !bf16ops;
  ki.scale2 = scale * scale;
  ki.nb_rows = pr.nb;
  ki.nb_cols = pr.nb;
  ki.rb_rows = pr.rb;
  ki.rbmax = bits_to_float(pr.st.rbmax_bits);
  ki.normmax = std::sqrt(bits_to_float(pr.st.nbmax_bits));
  ki.variant = P.screen_variant > 0 ? P.screen_variant - 1 : -1;
  TcShape tshape{-1, -1, -1, -1};
  // locality order of the screen's operands (speed only; the lists are exact either way)
  double ms_order = 0;
  if (screen == CNG_SCREEN_TC && !P.input_order) {
    st = apply_order(pool, &pr, dtype, n, d, dpad, kpad, &ki, &ms_order, s);
    if (st != CNG_OK) return st;
  }
  // integer data spanning <= 255: 8-bit rows for exact integer pair distances in the rerank
  // (K2), prune (K4) and merge (K6)
  uint8_t* u8 = nullptr;
  const int u8w = u8_rows_ok(pr.st, d) ? u8_words(d) : 0;
  if (u8w) {
    CK(pool.alloc(&u8, (size_t)n * u8w * 4));
    CK(launch_to_u8(pr.xs, dtype, n, d, dpad, key_to_float(pr.st.vmin_key), u8w, u8, s));
    ki.u8 = u8;
    ki.u8w = u8w;
  }
  double ms_screen = 0, ms_rerank = 0, ms_cand = 0;
  const bool beam = P.candidates == CNG_CAND_BEAM;
  const int K0 = P.knn_K > 0 ? P.knn_K : 200;
  int32_t* g0 = nullptr;  // beam route: G0 [n][K0]
  if (beam && P.knn_graph) {
    // the caller's G0 is checked before any search reads it
    g0 = const_cast<int32_t*>(P.knn_graph);
    uint32_t* gst;
    CK(pool.alloc(&gst, 1));
    CK(cudaMemsetAsync(gst, 0, 4, s));
    CK(launch_check_knn_graph(g0, n, K0, gst, s));
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, gst, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hst) return fail(CNG_E_INVAL, "knn_graph holds an id outside [0, n), a self edge or -1 before a neighbour");
  } else if (beam) {  // G0 = the exact K0-NN graph
    float* g0d;
    CK(pool.alloc(&g0, (size_t)n * K0));
    CK(pool.alloc(&g0d, (size_t)n * K0));
    KnnInputs kg = ki;
    kg.L = K0;
    kg.Lp = (int)std::min<int64_t>((int64_t)K0 + P.margin, n - 1);
    st = run_knn(kg, g0, g0d, ctr, &ms_screen, &ms_rerank, s, &tshape);
    if (st != CNG_OK) return st;
    cudaFree(g0d);
    pool.release(g0d);
  } else {
    st = run_knn(ki, cand, cdist, ctr, &ms_screen, &ms_rerank, s, &tshape);
    if (st != CNG_OK) return st;
  }
  // screening operands are no longer needed
  if (pr.tc) { cudaFree(pr.tc); pool.release(pr.tc); pr.tc = nullptr; }
  if (beam) {
    // Alg. 3 phase 2 (Sec. 4.1): beam search for every point on G0 from the navigating node;
    // its first L + 1 results hold the L closest visited points other than p
    const int Lb = P.beam_L > 0 ? P.beam_L : L + 1;
    Timer tc(s);
    tc.mark();
    int32_t h_entry0 = -1;
    CK(cudaMemcpyAsync(&h_entry0, d_entry, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    int32_t *qid, *deg0, *bid;
    float* bdist;
    int* bcounter;
    unsigned long long* btot;
    uint32_t* bstatus;
    CK(pool.alloc(&qid, (size_t)n));
    CK(pool.alloc(&deg0, (size_t)n));
    CK(pool.alloc(&bid, (size_t)n * (L + 1)));
    CK(pool.alloc(&bdist, (size_t)n * (L + 1)));
    CK(pool.alloc(&bcounter, SEARCH_COUNTER_INTS));
    CK(pool.alloc(&btot, 4));
    CK(pool.alloc(&bstatus, 1));
    CK(cudaMemsetAsync(bstatus, 0, 4, s));
    CK(launch_iota(qid, n, s));
    CK(launch_fill(deg0, n, K0, s));  // rows are -1 padded; the search reads the row alone
    CK(cudaStreamSynchronize(s));
    SearchArgs sa{};
    sa.X = pr.xs;
    sa.dtype = dtype;
    sa.n = n;
    sa.d = d;
    sa.dpad = dpad;
    sa.adj = g0;
    sa.deg = deg0;
    sa.R = K0;
    sa.entry = h_entry0;
    sa.qids = qid;
    sa.nq = n;
    sa.k = L + 1;
    sa.L = Lb;
    sa.band = band;
    sa.exact = exact;
    if (u8 && exact) {
      sa.U = u8;
      sa.u8w = u8w;
    }
    sa.counter = bcounter;
    sa.ids = bid;
    sa.dists = bdist;
    sa.tot = btot;
    sa.status = bstatus;
    SearchPlan plan;
    if (!search_plan(sa, 4, Lb <= 64 ? 1024 : 2048, &plan))
      return fail(CNG_E_UNSUPPORTED, "candidate search shape does not fit");
    CK(cudaMemsetAsync(bcounter, 0, SEARCH_COUNTER_INTS * sizeof(int), s));
    CK(launch_search(sa, plan, s));
    CK(launch_strip_self(bid, bdist, n, L, cand, cdist, &ctr->status, s));
    tc.mark();
    uint32_t sst = 0;
    CK(cudaMemcpyAsync(&sst, bstatus, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sst) return fail(CNG_E_INTERNAL, "candidate search exceeded n hop vertices");
    ms_cand = tc.ms(0, 1);
    cudaFree(bid);
    pool.release(bid);
    cudaFree(bdist);
    pool.release(bdist);
  }
  tm.mark();  // 3
  // phase 2b: prune every candidate list
  int32_t *fwd, *fdeg;
  CK(pool.alloc(&fwd, (size_t)n * R));
  CK(pool.alloc(&fdeg, (size_t)n));
  AlphaGrid ag{0.0, 0.0, -1};
  if (P.adaptive) {  // Alg. 4: i = 0 .. round((alpha_max - alpha0) / dalpha)
    ag.alpha0 = P.alpha0;
    ag.dalpha = P.dalpha;
    ag.imax = (int)std::floor((P.alpha_max - P.alpha0) / P.dalpha + 0.5);
  }
  float* half_norms = nullptr;  // FP16 rows on the Gram tile: |x|^2 per point
  if (!u8 && gram_prune_f16_ok(dtype, dpad, L, R, P.adaptive != 0))
    CK(pool.alloc(&half_norms, (size_t)n));
  CK(launch_prune_fwd(pr.xs, dtype, n, d, dpad, cand, cdist, L, P.alpha, P.tau, ag, R, band, fwd, fdeg,
                      ctr, u8, u8w, half_norms, s));
  tm.mark();  // 4
  // phase 3: reverse edges + lazy pruning
  int32_t *indeg, *cursor, *inl, *adj, *deg;
  int64_t *off, *bsum;
  CK(pool.alloc(&indeg, (size_t)n));
  CK(pool.alloc(&cursor, (size_t)n));
  CK(pool.alloc(&off, (size_t)n + 1));
  CK(pool.alloc(&bsum, (size_t)reverse_blocksums_len(n)));
  CK(pool.alloc(&inl, (size_t)n * R));
  const int Rs = R + (P.repair_slots > 0 ? P.repair_slots : REPAIR_SLOTS);
  CK(pool.alloc(&adj, (size_t)n * Rs));
  CK(pool.alloc(&deg, (size_t)n));
  int32_t* big_list;
  CK(pool.alloc(&big_list, 2 * (size_t)n));  // big list + the 8-bit merge's middle list
  CK(launch_reverse(fwd, fdeg, n, R, indeg, off, cursor, inl, bsum, ctr, s));
  MergeScratch ms{};  // merged sets listed for the Gram-tile (8-bit rows) or all-pairs re-prune
  if (!P.adaptive && (gram_prune_ok(u8, u8w, 128, R) || (!u8 && pairs_prune_ok(256, R, false)))) {
    ms.stride = u8 ? 128 : 256;
    CK(pool.alloc(&ms.mlist, (size_t)n * ms.stride));
    CK(pool.alloc(&ms.mdist, (size_t)n * ms.stride));
    CK(pool.alloc(&ms.mlen, (size_t)n));
    CK(pool.alloc(&ms.rlist, (size_t)n));
  }
  CK(launch_merge(pr.xs, dtype, n, d, dpad, fwd, fdeg, off, inl, P.alpha, P.tau, ag, R, band, exact, adj,
                  deg, Rs, ctr, big_list, u8, u8w, ms, s));
  {
    Counters hc0;
    CK(cudaMemcpyAsync(&hc0, ctr, sizeof(hc0), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hc0.nbig > 0) {  // hubs: merged sets above the shared-memory capacity
      int cap = 1;
      while (cap < R + hc0.max_indeg) cap <<= 1;
      int grid = std::min(hc0.nbig, num_sms() * 2);
      unsigned char* scratch;
      CK(pool.alloc(&scratch, (size_t)grid * cap * 17));
      CK(launch_merge_big(pr.xs, dtype, n, d, dpad, fwd, fdeg, off, inl, P.alpha, P.tau, ag, R, band,
                          exact, adj, deg, Rs, ctr, big_list, hc0.nbig, scratch, cap, grid, s));
    }
  }
  tm.mark();  // 5: merge done
  // phase 4: connectivity
  int32_t h_entry = -1;
  CK(cudaMemcpyAsync(&h_entry, d_entry, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int64_t repair_edges = 0;
  int repair_rounds = 0;
  if (P.connect_L >= 0) {
    const int Lc = P.connect_L > 0 ? P.connect_L : CONNECT_L;
    int32_t *reached, *fa, *fb, *U, *rid, *best, *rp, *has_in, *qdeg, *qhops;
    float* rdist;
    int* counts;
    int *sc_counter;
    unsigned long long* sc_tot;
    uint32_t* sc_status;
    CK(pool.alloc(&reached, (size_t)n));
    CK(pool.alloc(&fa, (size_t)n));
    CK(pool.alloc(&fb, (size_t)n));
    CK(pool.alloc(&U, (size_t)n));
    const int kc = Lc;  // every result of the search can name p
    CK(pool.alloc(&rid, (size_t)n * kc));
    CK(pool.alloc(&rdist, (size_t)n * kc));
    CK(pool.alloc(&best, (size_t)n));
    CK(pool.alloc(&rp, (size_t)n));
    CK(pool.alloc(&has_in, (size_t)n));
    CK(pool.alloc(&counts, 4));
    CK(pool.alloc(&sc_counter, SEARCH_COUNTER_INTS));
    CK(pool.alloc(&sc_tot, 4));
    CK(pool.alloc(&sc_status, 1));
    CK(cudaMemsetAsync(sc_status, 0, 4, s));
    (void)qdeg;
    (void)qhops;
    CK(launch_fill(best, n, 0x7fffffff, s));
    int hc_counts[4] = {0, 0, 0, 0};
    // rounds until every point is reachable (each adds at least one edge, else the phase
    // fails); the cap only bounds a pathological input
    constexpr int kMaxRounds = 4096;
    int round = 0;
    for (; round < kMaxRounds; ++round) {
      CK(launch_bfs(adj, deg, Rs, n, h_entry, reached, fa, fb, counts, hc_counts, s));
      CK(launch_collect(reached, n, U, counts + 2, s));
      CK(cudaMemcpyAsync(&hc_counts[2], counts + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const int nu = hc_counts[2];
      if (nu == 0) break;
      ++repair_rounds;
      SearchArgs sa{};
      sa.X = pr.xs;
      sa.dtype = dtype;
      sa.n = n;
      sa.d = d;
      sa.dpad = dpad;
      sa.adj = adj;
      sa.deg = deg;
      sa.R = Rs;
      sa.entry = h_entry;
      sa.Q = nullptr;
      sa.qids = U;
      sa.nq = nu;
      sa.k = kc;
      sa.L = Lc;
      sa.band = band;
      sa.exact = exact;
      if (u8 && exact) {  // stored points as queries: exact 8-bit rows
        sa.U = u8;
        sa.u8w = u8w;
      }
      sa.max_hops = 0;
      sa.counter = sc_counter;
      sa.ids = rid;
      sa.dists = rdist;
      sa.tot = sc_tot;
      sa.status = sc_status;
      SearchPlan plan;  // stored points are exact queries: nothing is deferred
      if (!search_plan(sa, 4, 1024, &plan))
        return fail(CNG_E_UNSUPPORTED, "connectivity search shape does not fit");
      CK(cudaMemsetAsync(sc_counter, 0, SEARCH_COUNTER_INTS * sizeof(int), s));
      CK(launch_search(sa, plan, s));
      // points without in-edges first (each edge necessary), several per row while its slots
      // last; else one edge per named row to the smallest point naming it
      CK(launch_has_in(adj, deg, Rs, n, has_in, s));
      CK(launch_pick(U, rid, nu, kc, deg, Rs, has_in, rp, counts + 3, s));
      CK(cudaMemcpyAsync(&hc_counts[3], counts + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const int zonly = hc_counts[3] > 0;
      int64_t added = 0;
      for (int step = 0; step <= Rs; ++step) {  // a row takes at most Rs edges
        CK(launch_claim_link(U, rp, nu, has_in, zonly, best, adj, deg, Rs, counts + 3, s));
        CK(cudaMemcpyAsync(&hc_counts[3], counts + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        added += hc_counts[3];
        if (!zonly || hc_counts[3] == 0) break;
      }
      if (added == 0)
        return fail(CNG_E_UNSUPPORTED, "phase 4 could not connect the graph (connectivity slots full; round " +
                                            std::to_string(round) + ", " + std::to_string(nu) +
                                            " points unreachable)");
      repair_edges += added;
    }
    if (round == kMaxRounds)
      return fail(CNG_E_UNSUPPORTED, "phase 4 did not connect the graph within " +
                                         std::to_string(kMaxRounds) + " rounds");
    uint32_t sst = 0;
    CK(cudaMemcpyAsync(&sst, sc_status, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (sst) return fail(CNG_E_INTERNAL, "connectivity search exceeded n hops");
  }
  tm.mark();  // 6: connectivity done
  Counters hc;
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  st = check_status(hc.status);
  if (st != CNG_OK) return st;

  cng_index* ix = new cng_index();
  ix->n = n;
  ix->d = d;
  ix->dpad = dpad;
  ix->dtype = dtype;
  ix->R = R;
  ix->rs = Rs;
  ix->L = L;
  ix->entry = h_entry;
  ix->exact = exact;
  ix->band = band;
  ix->xs = pr.xs;
  pool.release(pr.xs);
  ix->vmin = key_to_float(pr.st.vmin_key);
  ix->vmax = key_to_float(pr.st.vmax_key);
  if (u8) {
    ix->u8 = u8;
    ix->u8w = u8w;
    pool.release(u8);
  }
  ix->adj = adj;
  pool.release(adj);
  ix->deg = deg;
  pool.release(deg);
  if (P.keep_lists) {
    ix->cand = cand;
    pool.release(cand);
    ix->cdist = cdist;
    pool.release(cdist);
    ix->fwd = fwd;
    pool.release(fwd);
    ix->fdeg = fdeg;
    pool.release(fdeg);
  }
  if (cudaMalloc(&ix->counter, SEARCH_COUNTER_INTS * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ix->tot, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&ix->status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ix->status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ix->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ix->done, cudaEventDisableTiming) != cudaSuccess) {
    cng_free(ix);
    return fail(CNG_E_NOMEM, "index scratch allocation failed");
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->ms_total = tm.ms(0, 6);
    stats->ms_prep = tm.ms(0, 1);
    stats->ms_entry = tm.ms(1, 2);
    stats->ms_screen = ms_screen;
    stats->ms_rerank = ms_rerank;
    stats->ms_prune = tm.ms(3, 4);
    stats->ms_merge = tm.ms(4, 5);
    stats->ms_connect = tm.ms(5, 6);
    stats->n_edges = (int64_t)hc.edges + repair_edges;
    stats->repair_edges = repair_edges;
    stats->repair_rounds = repair_rounds;
    stats->screen_used = screen == CNG_SCREEN_TC && bf16ops ? CNG_SCREEN_TC_BF16 : screen;
    stats->cert_fail_rows = hc.nfail;
    stats->order_ties = (int64_t)hc.order_ties;
    stats->rule_ties = (int64_t)hc.rule_ties;
    stats->merge_repruned = (int64_t)hc.merge_repruned;
    stats->merge_max_list = std::max<int64_t>((int64_t)hc.merge_max_list, hc.max_indeg + R);
    stats->entry = h_entry;
    stats->exact_int = exact;
    stats->screen_err_max = bits_to_float(hc.screen_err_bits);
    stats->alpha_mean = P.adaptive ? P.alpha0 + P.dalpha * (double)hc.alpha_steps / (double)n
                                   : P.alpha;
    stats->ms_order = ms_order;
    stats->ms_cand_search = ms_cand;
    stats->screen_variant = tshape.variant;
    stats->screen_stages = tshape.stages;
    stats->screen_cap = tshape.cap;
    stats->screen_sync = tshape.sync_d;
    stats->prune_path = gram_prune_ok(u8, u8w, L, R)                 ? 2
                        : (u8 && L <= 256)                             ? 1
                        : half_norms                                   ? 3
                        : (!u8 && pairs_prune_ok(L, R, P.adaptive != 0)) ? 4
                                                                       : 0;
  }
  *out = ix;
  return CNG_OK;
}

extern "C" cng_status cng_graph(const cng_index* ix, const int32_t** adj, const int32_t** deg,
                                int32_t* R, int32_t* entry, int64_t* n) {
  if (!ix) return fail(CNG_E_INVAL, "index is NULL");
  if (adj) *adj = ix->adj;
  if (deg) *deg = ix->deg;
  if (R) *R = ix->rs;
  if (entry) *entry = ix->entry;
  if (n) *n = ix->n;
  return CNG_OK;
}

extern "C" cng_status cng_lists(const cng_index* ix, const int32_t** cand, const float** cdist,
                                int32_t* L, const int32_t** fwd, const int32_t** fdeg, int32_t* R) {
  if (!ix) return fail(CNG_E_INVAL, "index is NULL");
  if (!ix->cand) return fail(CNG_E_INVAL, "index was built without keep_lists");
  if (cand) *cand = ix->cand;
  if (cdist) *cdist = ix->cdist;
  if (L) *L = ix->L;
  if (fwd) *fwd = ix->fwd;
  if (fdeg) *fdeg = ix->fdeg;
  if (R) *R = ix->R;
  return CNG_OK;
}

// Exact data: per-query exactness flags and, with 8-bit rows, the queries as 8-bit rows
// (a buffer of the index, grown on demand; searches on one index run one at a time).
// The queries as the index searches them: device memory with the index's dimensions (host
// queries are copied; an inner-product index appends the zero coordinate).  Allocations are
// owned by `pool`.
static cng_status index_queries(const cng_index* ix, const float* queries, int64_t nq, DevPool& pool,
                                cudaStream_t s, const float** out) {
  const int din = ix->metric == CNG_IP ? ix->d - 1 : ix->d;
  const float* qd = queries;
  if (!is_device_ptr(queries)) {
    float* t;
    CK(pool.alloc(&t, (size_t)nq * din));
    CK(cudaMemcpyAsync(t, queries, (size_t)nq * din * 4, cudaMemcpyHostToDevice, s));
    qd = t;
  }
  if (ix->metric == CNG_IP) {
    float* a;
    CK(pool.alloc(&a, (size_t)nq * ix->d));
    CK(launch_append_zero(qd, nq, din, a, s));
    qd = a;
  }
  *out = qd;
  return CNG_OK;
}

// Grows the staging area of ix to at least `bytes` (callers hold ix->mu).
static cudaError_t ensure_stage(cng_index* ix, size_t bytes) {
  if (ix->stage_cap >= bytes) return cudaSuccess;
  cudaFree(ix->stage);
  ix->stage = nullptr;
  ix->stage_cap = 0;
  void* p = nullptr;
  size_t got = 0;
  const cudaError_t e = scratch_take(bytes, &p, &got);
  if (e == cudaSuccess) {
    ix->stage = static_cast<char*>(p);
    ix->stage_cap = got;
  }
  return e;
}

// Grows the deferred-query list of ix to at least nq entries (callers hold ix->mu).
static cudaError_t ensure_defer(cng_index* ix, int64_t nq) {
  if (ix->defer_cap >= nq) return cudaSuccess;
  cudaFree(ix->defer);
  ix->defer = nullptr;
  ix->defer_cap = 0;
  void* p = nullptr;
  size_t got = 0;
  const cudaError_t e = scratch_take((size_t)nq * sizeof(int32_t), &p, &got);
  if (e == cudaSuccess) {
    ix->defer = static_cast<int32_t*>(p);
    ix->defer_cap = (int64_t)(got / sizeof(int32_t));
  }
  return e;
}

// Orders this call after the index's previous one when they run on different streams (the
// per-index scratch -- queue counter, totals, status, query flags, deferred list, staging -- is
// shared by every call).  Callers hold ix->mu.
static cng_status order_after_last(cng_index* ix, cudaStream_t s) {
  if (ix->has_last && ix->last_stream != s) CK(cudaStreamWaitEvent(s, ix->done, 0));
  return CNG_OK;
}

static cng_status mark_done(cng_index* ix, cudaStream_t s) {
  CK(cudaEventRecord(ix->done, s));
  ix->last_stream = s;
  ix->has_last = true;
  return CNG_OK;
}

// Graphs cached per index (oldest evicted beyond this).
constexpr size_t MAX_GRAPHS = 16;

static cng_status search_queries(cng_index* ix, const float* qd, int64_t nq, SearchArgs* a,
                                 cudaStream_t s) {
  if (!ix->exact || ix->dtype != CNG_F32 || nq == 0) return CNG_OK;
  const size_t row = ix->u8 ? (size_t)ix->u8w * 4 : 0;
  const size_t need = ((size_t)nq + 15) / 16 * 16 + (size_t)nq * row;
  if (need > ix->qbuf_cap) {
    cudaFree(ix->qbuf);
    ix->qbuf = nullptr;
    ix->qbuf_cap = 0;
    CK(cudaMalloc(&ix->qbuf, need));
    ix->qbuf_cap = need;
  }
  uint8_t* flag = ix->qbuf;
  uint8_t* rows = ix->u8 ? ix->qbuf + ((size_t)nq + 15) / 16 * 16 : nullptr;
  CK(launch_query_check(qd, nq, ix->d, ix->vmin, ix->vmax, ix->u8w, rows, flag, s));
  a->qflag = flag;
  if (ix->u8) {
    a->U = ix->u8;
    a->QU = rows;
    a->u8w = ix->u8w;
  }
  return CNG_OK;
}

extern "C" cng_status cng_search(const cng_index* cix, const float* queries, int64_t nq, int32_t k,
                                 int32_t L, const cng_search_params* params, int32_t* ids,
                                 float* dists, int32_t* ndc, int32_t* hops, int32_t* flags,
                                 void* stream, cng_search_stats* stats) {
  cng_index* ix = const_cast<cng_index*>(cix);
  if (!ix) return fail(CNG_E_INVAL, "index must be non-NULL");
  if (nq < 0) return fail(CNG_E_INVAL, "nq must be >= 0");
  if (nq > 0 && (!queries || !ids || !dists))
    return fail(CNG_E_INVAL, "queries, ids and dists must be non-NULL when nq > 0");
  if (k < 1 || L < k || L > 256) return fail(CNG_E_INVAL, "need 1 <= k <= L <= 256");
  cng_search_params defp{};
  const cng_search_params& P = params ? *params : defp;
  if (P.mode != CNG_SEARCH_FIXED && P.mode != CNG_SEARCH_LEARNED) return fail(CNG_E_INVAL, "unknown mode");
  if (P.mode == CNG_SEARCH_LEARNED && (!P.model || !(P.threshold > 0.f && P.threshold < 1.f) || P.check_every < 1))
    return fail(CNG_E_INVAL, "learned mode needs a model, 0 < threshold < 1 and check_every >= 1");
  if (P.max_hops < 0) return fail(CNG_E_INVAL, "max_hops must be >= 0");
  if (P.min_stable < 0) return fail(CNG_E_INVAL, "min_stable must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  if (nq == 0) {
    if (stats) memset(stats, 0, sizeof(*stats));
    return CNG_OK;
  }
  // host queries / results and the inner-product queries go through the index's staging area,
  // so repeated host calls allocate nothing and keep their graph arguments
  const bool host_q = !is_device_ptr(queries);
  const bool host_out = !is_device_ptr(ids);
  {
    const void* outs[4] = {dists, ndc, hops, flags};
    const char* names[4] = {"dists", "ndc", "hops", "flags"};
    for (int i = 0; i < 4; ++i)
      if (outs[i] && is_device_ptr(outs[i]) == host_out)
        return fail(CNG_E_INVAL, std::string("outputs must all be host or all be device memory (ids is ") +
                                     (host_out ? "host" : "device") + ", " + names[i] + " is not)");
  }
  std::lock_guard<std::mutex> lock(ix->mu);
  {
    cng_status os = order_after_last(ix, s);
    if (os != CNG_OK) return os;
  }
  const int din = ix->metric == CNG_IP ? ix->d - 1 : ix->d;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  size_t need = 0;
  if (host_q) need += al((size_t)nq * din * 4);
  if (ix->metric == CNG_IP) need += al((size_t)nq * ix->d * 4);
  if (host_out)
    need += 2 * al((size_t)nq * k * 4) + (ndc ? al((size_t)nq * 4) : 0) +
            (hops ? al((size_t)nq * 4) : 0) + (flags ? al((size_t)nq * 4) : 0);
  CK(ensure_stage(ix, need));
  char* sp = ix->stage;
  auto carve = [&](size_t b) {
    char* r = sp;
    sp += al(b);
    return r;
  };
  const float* qd = queries;
  if (host_q) {
    float* t = reinterpret_cast<float*>(carve((size_t)nq * din * 4));
    CK(cudaMemcpyAsync(t, queries, (size_t)nq * din * 4, cudaMemcpyHostToDevice, s));
    qd = t;
  }
  if (ix->metric == CNG_IP) {
    float* t = reinterpret_cast<float*>(carve((size_t)nq * ix->d * 4));
    CK(launch_append_zero(qd, nq, din, t, s));
    qd = t;
  }
  int32_t *o_ids = ids, *o_ndc = ndc, *o_hops = hops, *o_flags = flags;
  float* o_d = dists;
  if (host_out) {
    o_ids = reinterpret_cast<int32_t*>(carve((size_t)nq * k * 4));
    o_d = reinterpret_cast<float*>(carve((size_t)nq * k * 4));
    if (ndc) o_ndc = reinterpret_cast<int32_t*>(carve((size_t)nq * 4));
    if (hops) o_hops = reinterpret_cast<int32_t*>(carve((size_t)nq * 4));
    if (flags) o_flags = reinterpret_cast<int32_t*>(carve((size_t)nq * 4));
  }
  SearchArgs a{};
  a.X = ix->xs;
  a.dtype = ix->dtype;
  a.n = ix->n;
  a.d = ix->d;
  a.dpad = ix->dpad;
  a.adj = ix->adj;
  a.deg = ix->deg;
  a.R = ix->rs;
  a.entry = ix->entry;
  a.Q = qd;
  a.nq = nq;
  a.k = k;
  a.L = L;
  a.band = ix->band;
  a.exact = ix->exact;
  a.max_hops = P.max_hops;
  a.counter = ix->counter;
  a.ids = o_ids;
  a.dists = o_d;
  a.ndc = o_ndc;
  a.hops = o_hops;
  a.flags = o_flags;
  a.tot = ix->tot;
  a.status = ix->status;
  if (P.mode == CNG_SEARCH_LEARNED) {
    a.model = P.model->blk;
    a.zthr = std::log(P.threshold / (1.f - P.threshold));
    a.check_every = P.check_every;
    a.min_stable = P.min_stable;
  }
  {
    cng_status qs = search_queries(ix, qd, nq, &a, s);
    if (qs != CNG_OK) return qs;
  }
  CK(ensure_defer(ix, nq));
  a.defer = ix->defer;
  SearchPlan plan;
  int wpb, hash;
  if (P.warps_per_block > 0) {  // caller's queries per CTA, default visited-filter size
    wpb = std::min(P.warps_per_block, 8);
    hash = L <= 64 ? 1024 : 2048;
    while (wpb > 1 && !search_plan(a, wpb, hash, &plan)) wpb >>= 1;
  } else {
    // autotune once per (L, mode): queries per CTA (warps per block) and visited-filter size,
    // each candidate timed on up to 16,384 of these queries; the results do not depend on it
    // (ids and hops are exact; only NDC varies with the lossy filter)
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> tl(g_tune_mu);
    auto it = std::find_if(g_tuned.begin(), g_tuned.end(), [&](const TunedShape& t) {
      return t.dev == dev && t.dtype == ix->dtype && t.dpad == ix->dpad && t.rs == ix->rs &&
             t.u8w == (a.U ? a.u8w : 0) && t.L == L && t.mode == P.mode;
    });
    if (it != g_tuned.end()) {
      wpb = it->wpb;
      hash = it->hash;
    } else {
      SearchArgs t = a;
      t.nq = std::min<int64_t>(nq, 16384);  // several waves, so the tail does not decide
      float best = 1e30f;
      wpb = 0;
      hash = 0;
      cudaEvent_t t0, t1;
      cudaEventCreate(&t0);
      cudaEventCreate(&t1);
      for (int h : {512, 1024, 2048}) {
        if (h < 2 * L) continue;
        for (int w : {1, 2, 4, 8}) {
          SearchPlan tp;
          if (!search_plan(t, w, h, &tp)) continue;
          float ms = 1e30f;
          for (int rep = 0; rep < 3; ++rep) {  // warm-up, then the faster of two timed runs
            CK(cudaMemsetAsync(ix->counter, 0, SEARCH_COUNTER_INTS * sizeof(int), s));
            cudaEventRecord(t0, s);
            CK(launch_search(t, tp, s));
            cudaEventRecord(t1, s);
            CK(cudaEventSynchronize(t1));
            float r = 0.f;
            cudaEventElapsedTime(&r, t0, t1);
            if (rep > 0) ms = std::min(ms, r);
          }
          if (ms < best) {
            best = ms;
            wpb = w;
            hash = h;
          }
        }
      }
      cudaEventDestroy(t0);
      cudaEventDestroy(t1);
      if (!wpb) return fail(CNG_E_UNSUPPORTED, "search shape does not fit in shared memory");
      g_tuned.push_back({dev, ix->dtype, ix->dpad, ix->rs, a.U ? a.u8w : 0, L, P.mode, wpb, hash});
    }
  }
  if (!search_plan(a, wpb, hash, &plan))
    return fail(CNG_E_UNSUPPORTED, "search shape does not fit in shared memory");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  CK(cudaMemsetAsync(ix->tot, 0, 4 * sizeof(unsigned long long), s));
  cudaEventRecord(e0, s);
  if (P.use_graph) {
    cudaGraphExec_t exec = nullptr;
    for (auto& g : ix->graphs)
      if (g.stream == s && !memcmp(&g.plan, &plan, sizeof(plan)) && !memcmp(&g.args, &a, sizeof(a)))
        exec = g.exec;
    if (!exec) {
      // capture on the index's private stream (the legacy default stream cannot be captured);
      // the instantiated graph is then launched on the caller's stream
      cudaGraph_t graph;
      cudaStream_t cs = ix->cap_stream;
      CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      cudaMemsetAsync(ix->counter, 0, SEARCH_COUNTER_INTS * sizeof(int), cs);
      launch_search(a, plan, cs);
      CK(cudaStreamEndCapture(cs, &graph));
      CK(cudaGraphInstantiate(&exec, graph, 0));
      cudaGraphDestroy(graph);
      if (ix->graphs.size() >= MAX_GRAPHS) {  // evict the oldest (earlier launches are queued)
        cudaGraphExecDestroy(ix->graphs.front().exec);
        ix->graphs.erase(ix->graphs.begin());
      }
      ix->graphs.push_back({a, plan, s, exec});
    }
    CK(cudaGraphLaunch(exec, s));
  } else {
    CK(cudaMemsetAsync(ix->counter, 0, SEARCH_COUNTER_INTS * sizeof(int), s));
    CK(launch_search(a, plan, s));
  }
  cudaEventRecord(e1, s);
  {
    cng_status ds = mark_done(ix, s);
    if (ds != CNG_OK) return ds;
  }
  if (host_out) {
    CK(cudaMemcpyAsync(ids, o_ids, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(dists, o_d, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s));
    if (ndc) CK(cudaMemcpyAsync(ndc, o_ndc, (size_t)nq * 4, cudaMemcpyDeviceToHost, s));
    if (hops) CK(cudaMemcpyAsync(hops, o_hops, (size_t)nq * 4, cudaMemcpyDeviceToHost, s));
    if (flags) CK(cudaMemcpyAsync(flags, o_flags, (size_t)nq * 4, cudaMemcpyDeviceToHost, s));
  }
  if (stats || host_out || host_q) {
    unsigned long long tot[4];
    uint32_t dst = 0;
    CK(cudaMemcpyAsync(tot, ix->tot, sizeof(tot), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&dst, ix->status, sizeof(dst), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (dst) {
      cudaMemsetAsync(ix->status, 0, sizeof(uint32_t), s);
      return fail(CNG_E_INTERNAL, "search exceeded n hop vertices (corrupted queue)");
    }
    if (stats) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      stats->ms = ms;
      stats->ndc_total = (int64_t)tot[0];
      stats->hops_total = (int64_t)tot[1];
      stats->fp64_decisions = (int64_t)tot[2];
      stats->stopped_early = (int64_t)tot[3];
      stats->warps_per_block = wpb;
      stats->hash_slots = hash;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  return CNG_OK;
}

extern "C" cng_status cng_tune_tau(const void* points, int32_t dtype, int64_t n, int32_t d,
                                   const cng_build_params* params, const float* queries,
                                   int64_t nq, int32_t k, const int32_t* gt_ids,
                                   const int32_t* search_Ls, int32_t n_Ls, double target,
                                   void* stream, double* best_tau, cng_tau_trial* trials,
                                   int32_t max_trials, int32_t* n_trials) {
  if (!points || !params || !queries || !gt_ids || !search_Ls || !best_tau || !n_trials)
    return fail(CNG_E_INVAL, "pointers must be non-NULL");
  if (nq < 1 || k < 1 || n_Ls < 1 || !(target > 0.0 && target <= 1.0) || max_trials < 0 ||
      (max_trials > 0 && !trials))
    return fail(CNG_E_INVAL, "need nq >= 1, k >= 1, n_Ls >= 1, 0 < target <= 1");
  for (int i = 0; i < n_Ls; ++i)
    if (search_Ls[i] < k || search_Ls[i] > 256 || (i > 0 && search_Ls[i] <= search_Ls[i - 1]))
      return fail(CNG_E_INVAL, "search_Ls must ascend with k <= L <= 256");
  cudaStream_t s = (cudaStream_t)stream;
  DevPool pool;
  int32_t *ids_d, *hops_d;
  float* dists_d;
  CK(pool.alloc(&ids_d, (size_t)nq * k));
  CK(pool.alloc(&dists_d, (size_t)nq * k));
  CK(pool.alloc(&hops_d, (size_t)nq));
  std::vector<int32_t> ids((size_t)nq * k), hops((size_t)nq);
  std::vector<std::vector<int32_t>> gt((size_t)nq);
  for (int64_t q = 0; q < nq; ++q) {
    gt[q].assign(gt_ids + q * k, gt_ids + (q + 1) * k);
    std::sort(gt[q].begin(), gt[q].end());
  }
  std::vector<cng_tau_trial> done;
  auto run = [&](double tau) -> cng_status {
    for (const auto& t : done)
      if (t.tau == tau) return CNG_OK;
    cng_build_params bp = *params;
    bp.tau = tau;
    cng_index* ix = nullptr;
    cng_status st = cng_build(points, dtype, n, d, &bp, stream, &ix, nullptr);
    if (st != CNG_OK) return st;
    cng_tau_trial tr{tau, 0, 0.0, 0.0};
    for (int li = 0; li < n_Ls; ++li) {
      cng_search_params sp{};
      st = cng_search(ix, queries, nq, k, search_Ls[li], &sp, ids_d, dists_d, nullptr, hops_d,
                      nullptr, stream, nullptr);
      if (st != CNG_OK) break;
      if (cudaMemcpyAsync(ids.data(), ids_d, ids.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(hops.data(), hops_d, hops.size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        st = fail(CNG_E_CUDA, "tau search: copy of the results failed");
        break;
      }
      double rec = 0.0, h = 0.0;
      for (int64_t q = 0; q < nq; ++q) {
        int hit = 0;
        for (int j = 0; j < k; ++j)
          hit += std::binary_search(gt[q].begin(), gt[q].end(), ids[q * k + j]) ? 1 : 0;
        rec += (double)hit / k;
        h += hops[q];
      }
      tr.recall = rec / (double)nq;
      tr.hops_mean = h / (double)nq;
      if (tr.recall >= target) {
        tr.L = search_Ls[li];
        break;
      }
    }
    cng_free(ix);
    if (st != CNG_OK) return st;
    done.push_back(tr);
    return CNG_OK;
  };
  // the better of two trials: reaches the target, then fewer hops, then smaller tau
  auto better = [](const cng_tau_trial& a, const cng_tau_trial& b) {
    if ((a.L > 0) != (b.L > 0)) return a.L > 0;
    if (a.L > 0 && a.hops_mean != b.hops_mean) return a.hops_mean < b.hops_mean;
    return a.tau < b.tau;
  };
  for (double tau : {0.0, 10.0, 1.0, 0.1, 0.01, 0.001}) {
    cng_status st = run(tau);
    if (st != CNG_OK) return st;
  }
  cng_tau_trial best = done[0];
  for (const auto& t : done)
    if (better(t, best)) best = t;
  const double fine[2] = {best.tau > 0.0 ? best.tau / 2 : 0.0005, best.tau > 0.0 ? best.tau * 2 : 0.0005};
  for (double tau : fine) {
    cng_status st = run(tau);
    if (st != CNG_OK) return st;
  }
  for (const auto& t : done)
    if (better(t, best)) best = t;
  *best_tau = best.L > 0 ? best.tau : 0.0;
  *n_trials = (int32_t)std::min<size_t>(done.size(), (size_t)max_trials);
  for (int i = 0; i < *n_trials; ++i) trials[i] = done[i];
  return CNG_OK;
}

extern "C" cng_status cng_knn(const float* base, int64_t n, const float* rows, int64_t m, int32_t d,
                              int32_t k, int32_t screen, double tie_band, int32_t* ids, float* dists,
                              void* stream, cng_build_stats* stats) {
  if (!base || !ids || !dists) return fail(CNG_E_INVAL, "base, ids and dists must be non-NULL");
  if (d < 1 || d > 4096) return fail(CNG_E_INVAL, "d must be in [1, 4096]");
  const bool self = rows == nullptr;
  if (self) m = n;
  if (n < 1 || m < 0 || k < 1 || k > 256 || k > n || (self && k >= n))
    return fail(CNG_E_INVAL, "need 1 <= k <= 256, k <= n (k < n without rows)");
  if (screen != CNG_SCREEN_FP32 && screen != CNG_SCREEN_TC && screen != CNG_SCREEN_TC_BF16)
    return fail(CNG_E_INVAL, "unknown screen");
  const int bf16ops = screen == CNG_SCREEN_TC_BF16;
  if (bf16ops) screen = CNG_SCREEN_TC;
  if (!(tie_band >= 5e-6) || tie_band > 0.01) return fail(CNG_E_INVAL, "tie_band must be in [5e-6, 0.01]");
  if (!is_device_ptr(base) || (!self && !is_device_ptr(rows)) || !is_device_ptr(ids) || !is_device_ptr(dists))
    return fail(CNG_E_INVAL, "cng_knn takes device pointers");
  if (m == 0) return CNG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (screen == CNG_SCREEN_TC && !tc_screen_supported(d, false)) screen = CNG_SCREEN_FP32;
  DevPool pool;
  const int dpad = round_up(d, 32), kpad = round_up(d, 64);
  Prepared pb, prw;
  float scale = 1.f;
  if (screen == CNG_SCREEN_TC && !bf16ops) {  // one scale for rows and columns
    const void* pl[2] = {base, rows};
    const int64_t nl[2] = {n, self ? 0 : m};
    cng_status ss = operand_scale(pl, nl, 2, CNG_F32, d, &scale, s);
    if (ss != CNG_OK) return ss;
  }
  cng_status st = prepare(pool, base, CNG_F32, n, d, dpad, screen, kpad, &pb, s, !bf16ops, scale);
  if (st != CNG_OK) return st;
  if (!self) {
    st = prepare(pool, rows, CNG_F32, m, d, dpad, screen, kpad, &prw, s, !bf16ops, scale);
    if (st != CNG_OK) return st;
  }
  Prepared& pr = self ? pb : prw;
  PrepStats both = pb.st;
  if (!self) {
    both.nonint |= prw.st.nonint;
    both.vmin_key = std::min(both.vmin_key, prw.st.vmin_key);
    both.vmax_key = std::max(both.vmax_key, prw.st.vmax_key);
    both.normmax_bits = std::max(both.normmax_bits, prw.st.normmax_bits);
    both.nbmax_bits = std::max(both.nbmax_bits, prw.st.nbmax_bits);
    both.rbmax_bits = std::max(both.rbmax_bits, prw.st.rbmax_bits);
  }
  Counters* ctr;
  CK(pool.alloc(&ctr, 1));
  CK(cudaMemsetAsync(ctr, 0, sizeof(Counters), s));
  KnnInputs ki{};
  ki.xr = pr.xs;
  ki.xc = pb.xs;
  ki.m = m;
  ki.n = n;
  ki.d = d;
  ki.dpad = dpad;
  ki.dtype = CNG_F32;
  ki.self_excl = self;
  ki.L = k;
  ki.Lp = (int)std::min<int64_t>((int64_t)k + 32, self ? n - 1 : n);
  ki.screen = screen;
  ki.band = (float)tie_band;
  ki.exact = exact_int(both, d, screen, bf16ops);
  ki.tc_rows = pr.tc;
  ki.tc_cols = pb.tc;
  ki.kpad = kpad;
  ki.tc_fp16 = !bf16ops;
  ki.scale2 = scale * scale;
  ki.nb_rows = pr.nb;
  ki.nb_cols = pb.nb;
  ki.rb_rows = pr.rb;
  ki.rbmax = bits_to_float(both.rbmax_bits);
  ki.normmax = std::sqrt(bits_to_float(both.nbmax_bits));
  double ms_order = 0;
  if (self && screen == CNG_SCREEN_TC) {
    st = apply_order(pool, &pb, CNG_F32, n, d, dpad, kpad, &ki, &ms_order, s);
    if (st != CNG_OK) return st;
  }
  double ms_screen = 0, ms_rerank = 0;
  st = run_knn(ki, ids, dists, ctr, &ms_screen, &ms_rerank, s);
  if (st != CNG_OK) return st;
  Counters hc;
  CK(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  st = check_status(hc.status);
  if (st != CNG_OK) return st;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->ms_screen = ms_screen;
    stats->ms_rerank = ms_rerank;
    stats->ms_total = ms_order + ms_screen + ms_rerank;
    stats->ms_order = ms_order;
    stats->cert_fail_rows = hc.nfail;
    stats->order_ties = (int64_t)hc.order_ties;
    stats->exact_int = ki.exact;
    stats->screen_used = screen == CNG_SCREEN_TC && bf16ops ? CNG_SCREEN_TC_BF16 : screen;
  }
  return CNG_OK;
}

static cng_status tc_scores(const float* rows, int64_t m, const float* cols, int64_t n, int32_t d,
                            int fp16, float scale, float* scores, void* stream) {
  if (!rows || !cols || !scores) return fail(CNG_E_INVAL, "pointers must be non-NULL");
  if (m < 1 || n < 1 || d < 1 || !tc_screen_supported(d, false))
    return fail(CNG_E_INVAL, "need m, n >= 1 and 1 <= d <= 4096");
  if (!(scale > 0.f) || std::ilogb(scale) != std::log2(scale))
    return fail(CNG_E_INVAL, "scale must be a power of two");
  cudaStream_t s = (cudaStream_t)stream;
  DevPool pool;
  const int dpad = round_up(d, 32), kpad = round_up(d, 64);
  Prepared pr, pc;
  cng_status st = prepare(pool, rows, CNG_F32, m, d, dpad, CNG_SCREEN_TC, kpad, &pr, s, fp16, scale);
  if (st != CNG_OK) return st;
  st = prepare(pool, cols, CNG_F32, n, d, dpad, CNG_SCREEN_TC, kpad, &pc, s, fp16, scale);
  if (st != CNG_OK) return st;
  uint32_t* status;
  CK(pool.alloc(&status, 1));
  CK(cudaMemsetAsync(status, 0, 4, s));
  TcScreenArgs ta{};
  ta.A = pr.tc;
  ta.B = pc.tc;
  ta.m = m;
  ta.n = n;
  ta.kpad = kpad;
  ta.fp16 = fp16;
  ta.nb = pc.nb;
  ta.Lp = 32;
  ta.self_excl = 0;
  ta.status = status;
  ta.rowbuf_words = screen_tc_rowbuf_words(m, n, 32);
  CK(pool.alloc(&ta.rowbuf, ta.rowbuf_words));
  std::string msg;
  cudaError_t e = launch_screen_tc_dump(ta, scores, s, &msg);
  if (e != cudaSuccess) return fail(CNG_E_CUDA, "tensor-core screen: " + msg + cudaGetErrorString(e));
  uint32_t hs = 0;
  CK(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return check_status(hs);
}

extern "C" cng_status cngx_tc_scores(const float* rows, int64_t m, const float* cols, int64_t n,
                                     int32_t d, float* scores, void* stream) {
  return tc_scores(rows, m, cols, n, d, 0, 1.f, scores, stream);
}

extern "C" cng_status cngx_wait_probe(uint32_t* status_out) {
  if (!status_out) return fail(CNG_E_INVAL, "status_out must be non-NULL");
  uint32_t* dev = nullptr;
  CK(cudaMalloc(&dev, 2 * sizeof(uint32_t)));
  cudaError_t e = cudaMemset(dev, 0, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) e = launch_wait_probe(dev, dev + 1, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status_out, dev, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(dev);
  CK(e);
  return CNG_OK;
}

extern "C" cng_status cngx_tc_scores_f16(const float* rows, int64_t m, const float* cols, int64_t n,
                                         int32_t d, float scale, float* scores, void* stream) {
  return tc_scores(rows, m, cols, n, d, 1, scale, scores, stream);
}


// ---------------------------------------------------------------------------------------------
// learned early stop
// ---------------------------------------------------------------------------------------------
__global__ void count_pos_kernel(const float* __restrict__ y, int64_t N, unsigned long long* c) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    m += y[i] > 0.5f;
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(c, m);
}

static cng_status new_model(cng_stop_model** out) {
  cng_stop_model* m = new cng_stop_model();
  if (cudaMalloc(&m->P, MLP_NPARAMS * 4) != cudaSuccess || cudaMalloc(&m->mu, 64) != cudaSuccess ||
      cudaMalloc(&m->sg, 64) != cudaSuccess || cudaMalloc(&m->blk, STOP_BLOCK_BYTES) != cudaSuccess) {
    cng_stop_free(m);
    return fail(CNG_E_NOMEM, "model allocation failed");
  }
  *out = m;
  return CNG_OK;
}

// Plain search with per-hop features (shared by cng_trace and cng_stop_train).
static cng_status run_trace(cng_index* ix, const float* qd, int64_t nq, int k, int L, int T,
                            float* feats, int32_t* hops, int32_t* tlc, int32_t* ids, float* dists,
                            cudaStream_t s) {
  SearchArgs a{};
  a.X = ix->xs;
  a.dtype = ix->dtype;
  a.n = ix->n;
  a.d = ix->d;
  a.dpad = ix->dpad;
  a.adj = ix->adj;
  a.deg = ix->deg;
  a.R = ix->rs;
  a.entry = ix->entry;
  a.Q = qd;
  a.nq = nq;
  a.k = k;
  a.L = L;
  a.band = ix->band;
  a.exact = ix->exact;
  a.counter = ix->counter;
  a.ids = ids;
  a.dists = dists;
  a.hops = hops;
  a.tlc = tlc;
  a.tot = ix->tot;
  a.status = ix->status;
  a.trace_feats = feats;
  a.max_trace = T;
  a.check_every = 1;
  cng_status qs = search_queries(ix, qd, nq, &a, s);  // callers hold ix->mu
  if (qs != CNG_OK) return qs;
  CK(ensure_defer(ix, nq));
  a.defer = ix->defer;
  SearchPlan plan;
  if (!search_plan(a, 4, L <= 64 ? 1024 : 2048, &plan))
    return fail(CNG_E_UNSUPPORTED, "search shape does not fit in shared memory");
  CK(cudaMemsetAsync(ix->counter, 0, SEARCH_COUNTER_INTS * sizeof(int), s));
  CK(launch_search(a, plan, s));
  return CNG_OK;
}

extern "C" cng_status cng_trace(const cng_index* cix, const float* queries, int64_t nq, int32_t k,
                                int32_t L, int32_t max_trace, float* feats, int32_t* hops,
                                int32_t* tlc, int32_t* ids, void* stream) {
  cng_index* ix = const_cast<cng_index*>(cix);
  if (!ix || !queries || !feats || !hops || !tlc || !ids) return fail(CNG_E_INVAL, "pointers must be non-NULL");
  if (nq < 1 || k < 1 || L < k || L > 256 || max_trace < 1) return fail(CNG_E_INVAL, "bad sizes");
  cudaStream_t s = (cudaStream_t)stream;
  DevPool pool;
  float* dists;
  CK(pool.alloc(&dists, (size_t)nq * k));
  const float* qd = nullptr;
  {
    cng_status qs = index_queries(ix, queries, nq, pool, s, &qd);
    if (qs != CNG_OK) return qs;
  }
  std::lock_guard<std::mutex> lock(ix->mu);
  cng_status st = order_after_last(ix, s);
  if (st == CNG_OK) st = run_trace(ix, qd, nq, k, L, max_trace, feats, hops, tlc, ids, dists, s);
  if (st == CNG_OK) st = mark_done(ix, s);
  if (st != CNG_OK) return st;
  CK(cudaStreamSynchronize(s));
  return CNG_OK;
}

extern "C" cng_status cng_stop_train(const cng_index* cix, const float* train_q, int64_t nq,
                                     const cng_train_params* params, void* stream,
                                     cng_stop_model** out, cng_train_stats* stats) {
  cng_index* ix = const_cast<cng_index*>(cix);
  if (!ix || !train_q || !params || !out) return fail(CNG_E_INVAL, "pointers must be non-NULL");
  *out = nullptr;
  const cng_train_params& P = *params;
  const int T = P.max_trace > 0 ? P.max_trace : 256;
  const int epochs = P.epochs > 0 ? P.epochs : 4;
  const int B = P.batch > 0 ? P.batch : 4096;
  const float lr = P.lr > 0.f ? P.lr : 1e-3f;
  if (nq < 1 || P.k < 1 || P.L < P.k || P.L > 256 || T > 4096 || B > (1 << 20))
    return fail(CNG_E_INVAL, "need nq >= 1, 1 <= k <= L <= 256, max_trace <= 4096, batch <= 2^20");
  cudaStream_t s = (cudaStream_t)stream;
  DevPool pool;
  const float* qd = nullptr;
  {
    cng_status qs = index_queries(ix, train_q, nq, pool, s, &qd);
    if (qs != CNG_OK) return qs;
  }
  Timer tm(s);
  tm.mark();
  float *feats, *dists;
  int32_t *hops, *tlc, *ids;
  int64_t* off;
  CK(pool.alloc(&feats, (size_t)nq * T * 16));
  CK(pool.alloc(&dists, (size_t)nq * P.k));
  CK(pool.alloc(&hops, (size_t)nq));
  CK(pool.alloc(&tlc, (size_t)nq));
  CK(pool.alloc(&ids, (size_t)nq * P.k));
  CK(pool.alloc(&off, (size_t)nq + 1));
  std::lock_guard<std::mutex> lock(ix->mu);
  cng_status st = order_after_last(ix, s);
  if (st == CNG_OK) st = run_trace(ix, qd, nq, P.k, P.L, T, feats, hops, tlc, ids, dists, s);
  if (st == CNG_OK) st = mark_done(ix, s);
  if (st != CNG_OK) return st;
  CK(launch_offsets(hops, nq, T, off, s));
  int64_t N = 0;
  CK(cudaMemcpyAsync(&N, off + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  tm.mark();
  if (N < 1) return fail(CNG_E_INVAL, "traces produced no samples");
  float *X, *y, *part, *ploss, *grad, *loss, *m, *v;
  double* spart;
  unsigned long long* npos;
  CK(pool.alloc(&X, (size_t)N * 16));
  CK(pool.alloc(&y, (size_t)N));
  CK(pool.alloc(&spart, 64 * 32));
  CK(pool.alloc(&npos, 1));
  const int Bn = (int)std::min<int64_t>(B, N);
  CK(pool.alloc(&part, (size_t)mlp_parts(Bn) * MLP_NPARAMS));
  CK(pool.alloc(&ploss, (size_t)mlp_parts(Bn)));
  CK(pool.alloc(&grad, MLP_NPARAMS));
  CK(pool.alloc(&loss, 2));
  CK(pool.alloc(&m, MLP_NPARAMS));
  CK(pool.alloc(&v, MLP_NPARAMS));
  cng_stop_model* mdl = nullptr;
  st = new_model(&mdl);
  if (st != CNG_OK) return st;
  auto guard = [&](cng_status r) {
    if (r != CNG_OK) cng_stop_free(mdl);
    return r;
  };
#define CKM(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return guard(fail(CNG_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  CKM(launch_samples(feats, hops, tlc, nq, T, off, X, y, s));
  CKM(cudaMemsetAsync(npos, 0, 8, s));
  count_launch();
  count_pos_kernel<<<num_sms() * 4, 256, 0, s>>>(y, N, npos);
  CKM(launch_standardise(X, N, spart, mdl->mu, mdl->sg, s));
  CKM(launch_mlp_init(mdl->P, P.seed ? P.seed : 1, s));
  CKM(cudaMemsetAsync(m, 0, MLP_NPARAMS * 4, s));
  CKM(cudaMemsetAsync(v, 0, MLP_NPARAMS * 4, s));
  const int64_t steps = std::max<int64_t>(1, (int64_t)epochs * ((N + Bn - 1) / Bn));
  const uint64_t seed = (P.seed ? P.seed : 1) * 0x2545F4914F6CDD1Dull + 7;
  for (int64_t t = 1; t <= steps; ++t) {
    float* lp = (t == 1) ? loss : (t == steps ? loss + 1 : nullptr);
    CKM(launch_mlp_grad(mdl->P, X, y, N, Bn, seed, t, part, ploss, grad, lp, s));
    CKM(launch_adam(mdl->P, m, v, grad, t, lr, s));
  }
  CKM(launch_pack_model(mdl->P, mdl->mu, mdl->sg, mdl->blk, s));
  tm.mark();
  float hl[2] = {0, 0};
  unsigned long long hp = 0;
  CKM(cudaMemcpyAsync(hl, loss, 8, cudaMemcpyDeviceToHost, s));
  CKM(cudaMemcpyAsync(&hp, npos, 8, cudaMemcpyDeviceToHost, s));
  CKM(cudaStreamSynchronize(s));
#undef CKM
  if (stats) {
    stats->ms_trace = tm.ms(0, 1);
    stats->ms_train = tm.ms(1, 2);
    stats->samples = N;
    stats->positives = (int64_t)hp;
    stats->steps = steps;
    stats->loss_first = hl[0];
    stats->loss_last = steps == 1 ? hl[0] : hl[1];
  }
  *out = mdl;
  return CNG_OK;
}

__global__ void bf16_round_kernel(const float* __restrict__ a, float* __restrict__ b, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __bfloat162float(__float2bfloat16_rn(a[i]));
}

extern "C" cng_status cng_stop_export(const cng_stop_model* m, float* params, float* mu, float* sigma,
                                      float* bf16_params) {
  if (!m) return fail(CNG_E_INVAL, "model is NULL");
  if (params) CK(cudaMemcpy(params, m->P, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost));
  if (mu) CK(cudaMemcpy(mu, m->mu, 64, cudaMemcpyDeviceToHost));
  if (sigma) CK(cudaMemcpy(sigma, m->sg, 64, cudaMemcpyDeviceToHost));
  if (bf16_params) {
    DevPool pool;
    float* t;
    CK(pool.alloc(&t, MLP_NPARAMS));
    count_launch();
    bf16_round_kernel<<<(MLP_NPARAMS + 255) / 256, 256>>>(m->P, t, MLP_NPARAMS);
    // weights are rounded for inference; biases, w3 and b3 stay FP32
    CK(cudaMemcpy(bf16_params, t, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost));
    float* full = new float[MLP_NPARAMS];
    cudaMemcpy(full, m->P, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost);
    const int b1 = 64 * 16, W2 = b1 + 64, b2 = W2 + 64 * 64;
    for (int i = b1; i < W2; ++i) bf16_params[i] = full[i];
    for (int i = b2; i < MLP_NPARAMS; ++i) bf16_params[i] = full[i];
    delete[] full;
  }
  return CNG_OK;
}

extern "C" cng_status cng_stop_import(const float* params, const float* mu, const float* sigma,
                                      cng_stop_model** out) {
  if (!params || !mu || !sigma || !out) return fail(CNG_E_INVAL, "pointers must be non-NULL");
  cng_stop_model* m = nullptr;
  cng_status st = new_model(&m);
  if (st != CNG_OK) return st;
  if (cudaMemcpy(m->P, params, MLP_NPARAMS * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->mu, mu, 64, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->sg, sigma, 64, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_pack_model(m->P, m->mu, m->sg, m->blk, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cng_stop_free(m);
    return fail(CNG_E_CUDA, "model upload failed");
  }
  *out = m;
  return CNG_OK;
}

extern "C" cng_status cng_mlp_grad(const float* params, const float* x, const float* y, int64_t B,
                                   float* grad, float* loss, void* stream) {
  if (!params || !x || !y || !grad) return fail(CNG_E_INVAL, "pointers must be non-NULL");
  if (B < 1 || B > (1 << 22)) return fail(CNG_E_INVAL, "B must be in [1, 2^22]");
  cudaStream_t s = (cudaStream_t)stream;
  DevPool pool;
  float *part, *ploss, *l;
  CK(pool.alloc(&part, (size_t)mlp_parts((int)B) * MLP_NPARAMS));
  CK(pool.alloc(&ploss, (size_t)mlp_parts((int)B)));
  CK(pool.alloc(&l, 1));
  CK(launch_mlp_grad(params, x, y, B, (int)B, 0, 0, part, ploss, grad, l, s));
  if (loss) CK(cudaMemcpyAsync(loss, l, 4, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  return CNG_OK;
}

extern "C" cng_status cng_mlp_adam(float* params, float* m, float* v, const float* grad, int64_t t,
                                   float lr, void* stream) {
  if (!params || !m || !v || !grad || t < 1) return fail(CNG_E_INVAL, "bad arguments");
  CK(launch_adam(params, m, v, grad, t, lr, (cudaStream_t)stream));
  return CNG_OK;
}

extern "C" long long cngx_launches(void) { return launch_counter().load(); }
