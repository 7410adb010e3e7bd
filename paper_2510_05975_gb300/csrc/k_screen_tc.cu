// k_screen_tc.cu -- tensor-core candidate screen (K1) for sm_103a: tcgen05.mma with TMEM
// accumulators, TMA tile loads into 128-byte-swizzled shared memory, mbarrier pipelines and
// a fused per-row top-L' filter.  It yields, for each row point x, a superset list of its
// nearest columns y by the screened score  s(x,y) = ||y_b||^2 - 2 <x_b, y_b>,  which differs
// from ||x_b - y_b||^2 only by the row constant ||x_b||^2 (x_b, y_b: bf16-rounded operands;
// fp16 operands for fp16 data).  The rerank (K2) recomputes FP32 distances and certifies
// the list; rows it cannot certify are rescanned exactly.
//
// CTA organisation (one CTA per SM, persistent over 256-row blocks):
//   warp 8      TMA producer: for kpad <= 192 the row block's A tile once, then B tiles of 128
//               columns with their column norms through an NST-stage ring (full / empty
//               mbarriers); for wider rows A and B together in 64-wide K chunks through the
//               same ring, and each tile's 128 column norms into a 4-slot norm ring
//   warp 9      TMEM owner (512 columns) and MMA issuer: per B tile, two M=128 x N=128
//               accumulators (rows 0-127 and 128-255), K in steps of 16, into one of two TMEM
//               buffers; tcgen05.commit frees each operand stage and publishes the buffer
//   warps 0-7   epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 of accumulator w / 4,
//               so each thread owns one row; 32 columns per tcgen05.ld; score = fma(-2, acc,
//               ||y_b||^2); the minimum of 32 scores is compared with the row threshold and
//               only then are entries appended to the row's buffer; full buffers are compacted
//               by the warp (radix select) which lowers the threshold
// All CTAs sweep the columns in the same order, so B tiles are shared through L2.
// Every mbarrier wait is bounded; on expiry the kernel records ST_TIMEOUT, drains its own
// TMA copies and MMAs (bounded) and frees TMEM before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "launch_count.h"
#include "cng_internal.h"
#include "device_common.cuh"
#include "screen_tc.h"

#include <mutex>
#include <vector>

namespace cng {

constexpr int TC_BM = 256;          // rows per CTA block (two M=128 accumulators)
constexpr int TC_BN = 128;          // columns per B tile
constexpr int TC_NBUF = 512 / (2 * TC_BN);  // accumulator buffers in the 512 TMEM columns
constexpr int TC_NBUF_LOG = TC_NBUF == 4 ? 2 : 1;
constexpr int TC_MAXST = TC_BN == 64 ? 8 : 4;  // operand stages at most
constexpr int TC_NR = 4;            // column-norm ring slots (tiles whose norms are in flight)
static_assert((2 * TC_MAXST + 2 * TC_NBUF + 2 * TC_NR + 3) * 8 + 8 <= 256,
              "barrier block exceeds its 256 bytes");
static_assert(TC_MAXST >= TC_NR, "the column-norm area holds max(stages, ring slots) tiles");
static_assert(TC_NBUF == 2 || TC_NBUF == 4, "two or four accumulator buffers");
constexpr int TC_KC = 64;           // K elements per 128-byte swizzle chunk
constexpr int TC_SLACK = 16;        // keys past the Lp-th a thinning may keep (one digit pass)
constexpr int TC_THREADS = 320;     // 8 epilogue warps + producer + MMA
constexpr int TC_PRODUCER = 8;
constexpr int TC_MMA = 9;
// wait iterations before declaring a timeout (each try_wait may suspend the thread for a
// system-dependent time; no suspend-time hint, so a completed phase is seen at once)
constexpr uint32_t TC_SPIN = 1u << 19;

struct TcParams {
  int64_t m, n;
  int kpad, nkc;        // kpad / 64
  int nst;              // B stages
  int Lp, cap, self_excl;
  uint32_t idesc;
  const float* nb;
  int32_t* ids;
  uint32_t* thr;
  uint64_t* rowbuf;
  uint32_t* status;
  const int32_t* perm;  // rows and columns are positions of a locality order: perm[pos] = id
  int wave_start;       // 1: each wave of row blocks starts its column sweep at its own rows
  int64_t row_off;      // position of row 0 in the order (a tuning trial on a row sample)
  uint32_t* sync;       // zeroed checkpoint counters (producers of a wave stay close), or null
  int sync_d;           // checkpoint lag in windows
};

// Producers meet at checkpoints every TC_SYNC_K tiles of their own sequence; a producer at
// checkpoint c waits until every CTA that reaches checkpoint c - sync_d has reached it, so
// the CTAs of a wave stay within sync_d * TC_SYNC_K B tiles of each other and share the tiles
// through L2 instead of each streaming them from DRAM.  The wait only serves the cache: it is
// bounded (about 2 ms) and the producer proceeds when it expires.
constexpr int TC_SYNC_K = 256 * 128 / TC_BN;  // tiles per checkpoint window (32,768 columns)
constexpr uint32_t TC_SYNC_SPIN = 8192;

CNG_DEV uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

CNG_DEV void wave_checkpoint(const TcParams& P, int64_t it, int64_t nrb, int ntiles) {
  if (!P.sync || it == 0 || it % TC_SYNC_K != 0) return;
  const int64_t c = it / TC_SYNC_K;
  atomicAdd(&P.sync[c], 1u);
  if (c <= P.sync_d) return;
  const int64_t cw = c - P.sync_d;
  // CTAs reaching tile index cw * K: those with a row block in wave (cw * K) / ntiles
  const int64_t w = (cw * TC_SYNC_K) / ntiles;
  const int64_t left = nrb - w * (int64_t)gridDim.x;
  const uint32_t expect = (uint32_t)(left < 0 ? 0 : (left > gridDim.x ? gridDim.x : left));
  for (uint32_t i = 0; i < TC_SYNC_SPIN; ++i) {
    if (ld_acquire_u32(&P.sync[cw]) >= expect) return;
    __nanosleep(200);
  }
}

// First column tile of row block rb's sweep.  A wave is the gridDim.x consecutive row blocks
// processed together; all its CTAs share the start, so B tiles stay shared through L2.
CNG_DEV int sweep_start(const TcParams& P, int64_t rb, int ntiles) {
  if (!P.wave_start) return 0;
  const int64_t w0 = rb - rb % gridDim.x;
  const int64_t t0 = (P.row_off + w0 * TC_BM) / TC_BN;
  return t0 < ntiles ? (int)t0 : ntiles - 1;
}

// ---- PTX wrappers ------------------------------------------------------------------------------
CNG_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

CNG_DEV void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
CNG_DEV void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
CNG_DEV void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
CNG_DEV bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false (and raises the CTA abort flag) on expiry or if aborted.
CNG_DEV bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, uint32_t* status) {
  for (uint32_t i = 0; i < TC_SPIN; ++i) {
    if (mbar_try(b, parity)) return true;
    if ((i & 15u) == 15u && *abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(status, ST_TIMEOUT);
  return false;
}

// Warp-uniform bounded wait: every lane polls, the warp proceeds only when all lanes saw the
// phase complete, so the whole warp leaves together (needed before .sync.aligned TMEM loads).
CNG_DEV bool mbar_wait_warp(uint64_t* b, uint32_t parity, volatile int* abort_flag, uint32_t* status,
                            uint32_t spin = TC_SPIN) {
  for (uint32_t i = 0; i < spin; ++i) {
    if (__all_sync(FULL, mbar_try(b, parity))) return true;
    if ((i & 15u) == 15u && __any_sync(FULL, *abort_flag != 0)) return false;
  }
  if ((threadIdx.x & 31) == 0) {
    *abort_flag = 1;
    atomicOr(status, ST_TIMEOUT);
  }
  __syncwarp();
  return false;
}

CNG_DEV void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

CNG_DEV void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms of 1024 B.
CNG_DEV uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // SWIZZLE_128B
  return d;
}

CNG_DEV void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
CNG_DEV void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
CNG_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
CNG_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

CNG_DEV void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

CNG_DEV void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Warp-cooperative selection (same contract as warp_compact): keeps the Lp smallest of the
// cnt buffered keys, moves them to the front and returns the largest kept key.  Radix select
// on 8-bit digits with a 256-bin shared histogram per warp (4 passes).
template <int CAP_PER_LANE>
CNG_DEV uint32_t warp_compact_hist(uint64_t* buf, int cnt, int Lp, int lane, uint32_t* hist) {
  uint32_t k[CAP_PER_LANE];
  uint64_t e[CAP_PER_LANE];
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) {
    int idx = i * 32 + lane;
    e[i] = idx < cnt ? buf[idx] : ~0ull;
    k[i] = (uint32_t)(e[i] >> 32);
  }
  __syncwarp();
  uint32_t prefix = 0;
  int need = Lp;
  const uint32_t hist_s = smem_u32(hist);
#pragma unroll 1
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < CAP_PER_LANE; ++i) {
      const bool valid = i * 32 + lane < cnt;
      const bool match = pass == 0 || ((k[i] ^ prefix) >> (shift + 8)) == 0;
      if (valid && match)
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(hist_s + 4u * ((k[i] >> shift) & 255u)) : "memory");
    }
    __syncwarp();
    uint32_t h[8], tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = hist[lane * 8 + i];
      tot += h[i];
    }
    uint32_t inc = tot;  // inclusive scan of lane totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - tot;
    const unsigned hit = __ballot_sync(FULL, excl < (uint32_t)need && inc >= (uint32_t)need);
    const int src = __ffs(hit) - 1;
    int digit = 0, below = 0;
    if (lane == src) {
      uint32_t acc = excl;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (acc + h[i] >= (uint32_t)need) { digit = lane * 8 + i; break; }
        acc += h[i];
      }
      below = (int)acc;
    }
    digit = __shfl_sync(FULL, digit, src);
    below = __shfl_sync(FULL, below, src);
    need -= below;
    prefix |= (uint32_t)digit << shift;
    __syncwarp();
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

// Warp-cooperative thinning of a row's buffer between tiles: keeps every buffered key up to a
// cut, with Lp <= kept <= Lp + slack, moves them to the front and returns the largest kept key
// (the row's new threshold); *kept = their number.  Each dropped key lies above every kept one,
// so at least Lp buffered keys stay at or below the threshold and no dropped column can be
// among the row's Lp smallest.  The radix select runs on the keys relative to the buffer's
// minimum, shifted left until the range fills 32 bits, so the first 8-bit digit already spans
// the buffer: one histogram pass usually places the cut (a bucket of at most `slack` keys past
// the Lp-th is kept whole).  Otherwise the next digit refines it, and after the last digit
// the ties at the Lp-th key are kept in buffer order as in warp_compact_hist.
template <int CAP_PER_LANE>
CNG_DEV uint32_t warp_thin_hist(uint64_t* buf, int cnt, int Lp, int slack, int lane, uint32_t* hist,
                                int* kept) {
  uint32_t k[CAP_PER_LANE];
  uint64_t e[CAP_PER_LANE];
  uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) {
    const int idx = i * 32 + lane;
    e[i] = idx < cnt ? buf[idx] : ~0ull;
    k[i] = (uint32_t)(e[i] >> 32);
    if (idx < cnt) {
      kmin = min(kmin, k[i]);
      kmax = max(kmax, k[i]);
    }
  }
  kmin = __reduce_min_sync(FULL, kmin);
  kmax = __reduce_max_sync(FULL, kmax);
  const uint32_t range = kmax - kmin;
  const int sh = range ? __clz(range) : 0;
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) k[i] = (k[i] - kmin) << sh;  // order kept: no overflow
  __syncwarp();
  uint32_t prefix = 0;
  int need = Lp, shift = 24;
  bool whole = false;
  const uint32_t hist_s = smem_u32(hist);
#pragma unroll 1
  for (int pass = 0; pass < 4; ++pass) {
    shift = 24 - 8 * pass;
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < CAP_PER_LANE; ++i) {
      const bool valid = i * 32 + lane < cnt;
      const bool match = pass == 0 || ((k[i] ^ prefix) >> (shift + 8)) == 0;
      if (valid && match)
        asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(hist_s + 4u * ((k[i] >> shift) & 255u)) : "memory");
    }
    __syncwarp();
    uint32_t h[8], tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      h[i] = hist[lane * 8 + i];
      tot += h[i];
    }
    uint32_t inc = tot;  // inclusive scan of lane totals
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - tot;
    const unsigned hit = __ballot_sync(FULL, excl < (uint32_t)need && inc >= (uint32_t)need);
    const int src = __ffs(hit) - 1;
    int digit = 0, below = 0, hd = 0;
    if (lane == src) {
      uint32_t acc = excl;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (acc + h[i] >= (uint32_t)need) {
          digit = lane * 8 + i;
          hd = (int)h[i];
          break;
        }
        acc += h[i];
      }
      below = (int)acc;
    }
    digit = __shfl_sync(FULL, digit, src);
    below = __shfl_sync(FULL, below, src);
    hd = __shfl_sync(FULL, hd, src);
    need -= below;  // keys still needed from the bucket `digit` (1 .. hd)
    prefix |= (uint32_t)digit << shift;
    __syncwarp();
    if (hd - need <= slack) {
      whole = true;
      break;
    }
  }
  // whole: keep every key up to the bucket's end; else keep the keys below prefix and the first
  // `need` equal to it
  const uint32_t cut = whole ? (prefix | ((1u << shift) - 1u)) : prefix;
  int out = 0, eq_taken = 0;
  uint32_t kmx = 0u;
#pragma unroll
  for (int i = 0; i < CAP_PER_LANE; ++i) {
    const bool valid = i * 32 + lane < cnt;
    const bool lt = valid && (whole ? k[i] <= cut : k[i] < cut);
    const bool eq = !whole && valid && k[i] == cut;
    const unsigned beq = __ballot_sync(FULL, eq);
    const int eq_rank = eq_taken + __popc(beq & ((1u << lane) - 1));
    const bool keep = lt || (eq && eq_rank < need);
    eq_taken += __popc(beq);
    const unsigned bk = __ballot_sync(FULL, keep);
    if (keep) {
      buf[out + __popc(bk & ((1u << lane) - 1))] = e[i];
      kmx = max(kmx, (uint32_t)(e[i] >> 32));
    }
    out += __popc(bk);
  }
  __syncwarp();
  *kept = out;
  return __reduce_max_sync(FULL, kmx);
}

CNG_DEV float min3f(float a, float b, float c) {
  float m;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
  return m;
}

// (a0, a1) * (b0, b1) + (c0, c1), each lane an IEEE fma rounded to nearest (same bits as fmaf)
CNG_DEV void fma2(uint32_t& d0, uint32_t& d1, uint32_t a0, uint32_t a1, float b, float c0, float c1) {
  uint64_t a, bb, c, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "r"(a0), "r"(a1));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
  asm("mov.b64 %0, {%1, %2};" : "=l"(c) : "f"(c0), "f"(c1));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(bb), "l"(c));
  asm("mov.b64 {%0, %1}, %2;" : "=r"(d0), "=r"(d1) : "l"(r));
}

CNG_DEV float4 lds_f4(uint32_t saddr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(saddr));
  return v;
}

CNG_DEV float fu(uint32_t x) { return __uint_as_float(x); }

// One row's 32 accumulator columns [cb, cb + 32): screened scores fma(-2, acc, ||y_b||^2) with
// the column norms from the norm ring (shared memory, the same address in every lane), masking
// of out-of-range and self columns, the minimum against the row threshold and appends below
// it.  The minimum is taken per group of 4 columns first, so appends visit only groups that
// hold one; every branch is warp-uniform.
template <bool DUMP>
CNG_DEV void process_chunk(uint32_t* r, int64_t cb, bool edge, bool live, int64_t row,
                           const TcParams& P, uint32_t nbs, float thr, int& cnt,
                           uint64_t* rbuf, float* dump) {
  float4 y[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) y[q] = lds_f4(nbs + 16 * q);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    fma2(r[4 * q + 0], r[4 * q + 1], r[4 * q + 0], r[4 * q + 1], -2.f, y[q].x, y[q].y);
    fma2(r[4 * q + 2], r[4 * q + 3], r[4 * q + 2], r[4 * q + 3], -2.f, y[q].z, y[q].w);
  }
  if (edge) {
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const int64_t col = cb + jj;
      if (col >= P.n || (P.self_excl && col == row)) r[jj] = 0x7f800000u;
    }
  }
  if constexpr (DUMP) {
    if (live)
#pragma unroll
      for (int jj = 0; jj < 32; ++jj)
        if (cb + jj < P.n) dump[row * P.n + cb + jj] = fu(r[jj]);
  } else {
    float gm[8];
#pragma unroll
    for (int g = 0; g < 8; ++g)
      gm[g] = fminf(min3f(fu(r[4 * g]), fu(r[4 * g + 1]), fu(r[4 * g + 2])), fu(r[4 * g + 3]));
    const float mall = min3f(min3f(gm[0], gm[1], gm[2]), min3f(gm[3], gm[4], gm[5]), fminf(gm[6], gm[7]));
    // appends, under warp-uniform branches (all lanes of the warp are converged here)
    const bool want = live && mall < thr;
    if (__any_sync(FULL, want)) {
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        const bool wg = want && gm[g] < thr;
        if (__any_sync(FULL, wg)) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float vj = fu(r[4 * g + k]);
            if (wg && vj < thr) {
              if (cnt < P.cap)
                rbuf[cnt] = ((uint64_t)fkey(vj) << 32) | (uint32_t)(cb + 4 * g + k);
              else
                atomicOr(P.status, ST_OVERFLOW);
              ++cnt;
            }
          }
        }
      }
    }
  }
}

// ---- the kernel --------------------------------------------------------------------------------
// KSTREAM = false: the row block's A tile stays resident (kpad <= 192) and each stage holds one
//   B tile of TC_BN columns x kpad.
// KSTREAM = true: A and B are streamed together in 64-wide K chunks (any kpad), each stage
//   holding the row block's A chunk and the column tile's B chunk; the accumulators sum the
//   chunks of a tile in TMEM.
template <int CPL, bool DUMP, bool KSTREAM>
__global__ void __launch_bounds__(TC_THREADS, 1)
screen_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 TcParams P, float* dump) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tile region
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = KSTREAM ? 0 : TC_BM * P.kpad * 2;
  const int stage_bytes = KSTREAM ? (TC_BM + TC_BN) * TC_KC * 2 : TC_BN * P.kpad * 2;
  unsigned char* sA = smem;
  unsigned char* sB = smem + a_bytes;
  // column norms: per operand stage with a resident A tile, else a TC_NR-slot ring
  float* sNB = reinterpret_cast<float*>(sB + P.nst * stage_bytes);  // [max(nst, TC_NR)][TC_BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>(sNB + TC_MAXST * TC_BN);
  uint64_t* b_full = bars;               // [nst]
  uint64_t* b_empty = bars + P.nst;      // [nst]
  uint64_t* t_full = bars + 2 * P.nst;   // [TC_NBUF]
  uint64_t* t_empty = t_full + TC_NBUF;  // [TC_NBUF]
  uint64_t* n_full = t_empty + TC_NBUF;  // [TC_NR]
  uint64_t* n_empty = n_full + TC_NR;    // [TC_NR]
  uint64_t* a_full = n_empty + TC_NR;    // [1]
  uint64_t* a_empty = a_full + 1;        // [1]
  uint64_t* fin = a_empty + 1;           // [1] MMA drain at exit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint32_t* hist_all = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(bars) + 256);  // [8][256]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nrb = (P.m + TC_BM - 1) / TC_BM;
  const int ntiles = (int)((P.n + TC_BN - 1) / TC_BN);

  if (tid == 0) {
    for (int i = 0; i < P.nst; ++i) {
      mbar_init(&b_full[i], 1);
      // the MMA's commit; with a resident A tile each stage also carries its tile's column
      // norms, which the 8 epilogue warps release
      mbar_init(&b_empty[i], KSTREAM ? 1 : 1 + 8);
    }
    for (int i = 0; i < TC_NBUF; ++i) {
      mbar_init(&t_full[i], 1);
      mbar_init(&t_empty[i], 8);
    }
    for (int i = 0; i < TC_NR; ++i) {
      mbar_init(&n_full[i], 1);
      mbar_init(&n_empty[i], 8);
    }
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == TC_PRODUCER) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
      int64_t it = 0;
      int j = 0;
      int s = 0;         // stage of the next copy (advanced without dividing)
      uint32_t ph = 0;   // its phase
      int ns = 0;        // norm ring slot of the next tile
      uint32_t nph = 0;  // its phase
      bool ok = true;
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, ++j) {
        if (!KSTREAM) {
          ok = mbar_wait(a_empty, (j & 1) ^ 1, abort_flag, P.status);
          if (!ok) break;
          mbar_expect_tx(a_full, (uint32_t)a_bytes);
          for (int kc = 0; kc < P.nkc; ++kc)
            tma_load_2d(sA + kc * (TC_BM * 128), &mapA, kc * TC_KC, (int)(rb * TC_BM), a_full);
        }
        const int t0 = sweep_start(P, rb, ntiles);
        for (int ti = 0; ti < ntiles; ++ti, ++it) {
          const int t = ti + t0 < ntiles ? ti + t0 : ti + t0 - ntiles;
          wave_checkpoint(P, it, nrb, ntiles);
          if (!KSTREAM) {
            // the B tile and its column norms into one stage
            ok = mbar_wait(&b_empty[s], ph ^ 1, abort_flag, P.status);
            if (!ok) break;
            mbar_expect_tx(&b_full[s], (uint32_t)(stage_bytes + TC_BN * 4));
            unsigned char* dst = sB + s * stage_bytes;
            for (int kc = 0; kc < P.nkc; ++kc)
              tma_load_2d(dst + kc * (TC_BN * 128), &mapB, kc * TC_KC, t * TC_BN, &b_full[s]);
            bulk_load(sNB + s * TC_BN, P.nb + (int64_t)t * TC_BN, TC_BN * 4, &b_full[s]);
            if (++s == P.nst) {
              s = 0;
              ph ^= 1u;
            }
          } else {
            // the tile's column norms into the norm ring, then A and B in K chunks
            ok = mbar_wait(&n_empty[ns], nph ^ 1, abort_flag, P.status);
            if (!ok) break;
            mbar_expect_tx(&n_full[ns], TC_BN * 4);
            bulk_load(sNB + ns * TC_BN, P.nb + (int64_t)t * TC_BN, TC_BN * 4, &n_full[ns]);
            if (++ns == TC_NR) {
              ns = 0;
              nph ^= 1u;
            }
            for (int kc = 0; kc < P.nkc && ok; ++kc) {
              ok = mbar_wait(&b_empty[s], ph ^ 1, abort_flag, P.status);
              if (!ok) break;
              mbar_expect_tx(&b_full[s], (uint32_t)stage_bytes);
              unsigned char* dst = sB + s * stage_bytes;
              tma_load_2d(dst, &mapA, kc * TC_KC, (int)(rb * TC_BM), &b_full[s]);
              tma_load_2d(dst + TC_BM * 128, &mapB, kc * TC_KC, t * TC_BN, &b_full[s]);
              if (++s == P.nst) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (!ok) break;
          }
        }
      }
      if (!ok) {
        // drain: wait (bounded) for copies this thread issued into stages not yet consumed
        for (int i = 0; i < P.nst; ++i) {
          for (uint32_t w = 0; w < (1u << 20); ++w)
            if (mbar_try(&b_full[i], 0) || mbar_try(&b_full[i], 1)) break;
        }
        for (int i = 0; i < TC_NR; ++i) {
          for (uint32_t w = 0; w < (1u << 20); ++w)
            if (mbar_try(&n_full[i], 0) || mbar_try(&n_full[i], 1)) break;
        }
      }
    }
  } else if (warp == TC_MMA) {
    if (lane == 0) {
      int64_t tt = 0;
      int j = 0;
      int s = 0;         // stage (advanced without dividing)
      uint32_t sph = 0;  // its phase
      bool ok = true;
      for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, ++j) {
        if (!KSTREAM) {
          ok = mbar_wait(a_full, j & 1, abort_flag, P.status);
          if (!ok) break;
          tc_fence_after();
        }
        const uint32_t a_base = smem_u32(sA);
        for (int t = 0; t < ntiles; ++t, ++tt) {
          const int b = (int)(tt & (TC_NBUF - 1));
          const uint32_t d_base = tmem + (uint32_t)(b * (2 * TC_BN));
          if (!KSTREAM) {
            ok = mbar_wait(&b_full[s], sph, abort_flag, P.status);
            if (!ok) break;
            ok = mbar_wait(&t_empty[b], (uint32_t)(((tt >> TC_NBUF_LOG) & 1) ^ 1), abort_flag, P.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t b_base = smem_u32(sB + s * stage_bytes);
            for (int kc = 0; kc < P.nkc; ++kc) {
#pragma unroll
              for (int k16 = 0; k16 < TC_KC / 16; ++k16) {
                const uint64_t bd = desc_sw128(b_base + kc * (TC_BN * 128) + k16 * 32);
#pragma unroll
                for (int acc = 0; acc < 2; ++acc) {
                  const uint64_t ad = desc_sw128(a_base + kc * (TC_BM * 128) + acc * (128 * 128) + k16 * 32);
                  mma_f16(d_base + (uint32_t)(acc * TC_BN), ad, bd, P.idesc, (kc | k16) != 0);
                }
              }
            }
            mma_commit(&b_empty[s]);
            if (++s == P.nst) {
              s = 0;
              sph ^= 1u;
            }
          } else {
            ok = mbar_wait(&t_empty[b], (uint32_t)(((tt >> TC_NBUF_LOG) & 1) ^ 1), abort_flag, P.status);
            if (!ok) break;
            for (int kc = 0; kc < P.nkc && ok; ++kc) {
              ok = mbar_wait(&b_full[s], sph, abort_flag, P.status);
              if (!ok) break;
              tc_fence_after();
              const uint32_t st_base = smem_u32(sB + s * stage_bytes);
#pragma unroll
              for (int k16 = 0; k16 < TC_KC / 16; ++k16) {
                const uint64_t bd = desc_sw128(st_base + TC_BM * 128 + k16 * 32);
#pragma unroll
                for (int acc = 0; acc < 2; ++acc) {
                  const uint64_t ad = desc_sw128(st_base + acc * (128 * 128) + k16 * 32);
                  mma_f16(d_base + (uint32_t)(acc * TC_BN), ad, bd, P.idesc, (kc | k16) != 0);
                }
              }
              mma_commit(&b_empty[s]);
              if (++s == P.nst) {
                s = 0;
                sph ^= 1u;
              }
            }
            if (!ok) break;
          }
          mma_commit(&t_full[b]);
        }
        if (!ok) break;
        if (!KSTREAM) mma_commit(a_empty);
      }
      // drain every MMA this thread issued before TMEM is released
      mma_commit(fin);
      for (uint32_t i = 0; i < (1u << 24); ++i)
        if (mbar_try(fin, 0)) break;
    }
  } else {
    // ---- epilogue: warps 0-7, one row per thread ----
    const int quarter = warp & 3, accsel = warp >> 2;
    const int rloc = accsel * 128 + quarter * 32 + lane;  // row within the block
    uint64_t* rbuf = P.rowbuf + ((size_t)blockIdx.x * TC_BM + rloc) * P.cap;
    uint32_t* hist = hist_all + warp * 256;
    int64_t tt = 0;
    int ns = 0;        // norm slot (stage, or ring slot) of tile tt, advanced without dividing
    uint32_t nph = 0;  // its phase
    bool ok = true;
    for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
      const int64_t row = rb * TC_BM + rloc;
      const bool live = row < P.m;
      float thr = __int_as_float(0x7f800000);
      int cnt = 0;
      const int t0 = sweep_start(P, rb, ntiles);
      for (int ti = 0; ti < ntiles; ++ti, ++tt) {
        const int t = ti + t0 < ntiles ? ti + t0 : ti + t0 - ntiles;
        const int b = (int)(tt & (TC_NBUF - 1));
        ok = mbar_wait_warp(&t_full[b], (uint32_t)((tt >> TC_NBUF_LOG) & 1), abort_flag, P.status);
        if (!ok) break;
        tc_fence_after();
        // the tile's column norms: the producer's copy (with the B stage, or into the ring
        // slot) is complete; the stage cannot be refilled before this warp releases it
        ok = KSTREAM ? mbar_wait_warp(&n_full[ns], nph, abort_flag, P.status)
                     : mbar_wait_warp(&b_full[ns], nph, abort_flag, P.status);
        if (!ok) break;
        const int64_t c0 = (int64_t)t * TC_BN;
        const bool edge = (c0 + TC_BN > P.n) || (P.self_excl && row >= c0 && row < c0 + TC_BN);
        const uint32_t ta =
            tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * (2 * TC_BN) + accsel * TC_BN);
#pragma unroll 1
        for (int ch = 0; ch < TC_BN / 32; ++ch) {
          uint32_t r[32];
          tmem_ld32_nowait(ta + ch * 32, r);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (ch == TC_BN / 32 - 1) {  // the last TMEM load of the tile: buffer back to the MMA
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[b]);
          }
          process_chunk<DUMP>(r, c0 + ch * 32, edge, live, row, P,
                              smem_u32(sNB + ns * TC_BN + ch * 32), thr, cnt, rbuf, dump);
        }
        // the norms of this slot (stage) are no longer needed: release it to the producer
        __syncwarp();
        if (lane == 0) mbar_arrive(KSTREAM ? &n_empty[ns] : &b_empty[ns]);
        if (++ns == (KSTREAM ? TC_NR : P.nst)) {
          ns = 0;
          nph ^= 1u;
        }
        if (DUMP) continue;
        // compact every row whose buffer could overflow on the next tile
        unsigned needc = __ballot_sync(FULL, cnt > P.cap - TC_BN);
        while (needc) {
          const int l = __ffs(needc) - 1;
          needc &= needc - 1;
          const int c_l = min(__shfl_sync(FULL, cnt, l), P.cap);
          uint64_t* buf_l = reinterpret_cast<uint64_t*>(__shfl_sync(FULL, reinterpret_cast<uintptr_t>(rbuf), l));
          __syncwarp();
          int kept;
          const uint32_t k = warp_thin_hist<CPL>(buf_l, c_l, P.Lp, TC_SLACK, lane, hist, &kept);
          if (lane == l) {
            thr = fkey_inv(k);
            cnt = kept;
          }
        }
      }
      if (!ok || DUMP) continue;
      // final: keep Lp per row, write ids and the threshold key
      uint32_t thk = fkey(thr);
      if (isinf(thr) && thr > 0.f) thk = 0xffffffffu;
      unsigned needf = __ballot_sync(FULL, cnt > P.Lp);
      while (needf) {
        const int l = __ffs(needf) - 1;
        needf &= needf - 1;
        const int c_l = min(__shfl_sync(FULL, cnt, l), P.cap);
        uint64_t* buf_l = reinterpret_cast<uint64_t*>(__shfl_sync(FULL, reinterpret_cast<uintptr_t>(rbuf), l));
        __syncwarp();
        const uint32_t k = warp_compact_hist<CPL>(buf_l, c_l, P.Lp, lane, hist);
        if (lane == l) {
          thk = k;
          cnt = P.Lp;
        }
      }
      __syncwarp();
      if (live) {
        const int c = min(cnt, P.Lp);
        const int64_t orow = P.perm ? P.perm[row] : row;
        for (int t = 0; t < P.Lp; ++t) {
          int32_t id = -1;
          if (t < c) id = P.perm ? P.perm[key_id(rbuf[t])] : key_id(rbuf[t]);
          P.ids[orow * P.Lp + t] = id;
        }
        P.thr[orow] = thk;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_MMA) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Failure-path probe: one warp waits, with the screen's own bounded wait, on an mbarrier that
// nothing arrives on (and, with spin_flag, on a global flag nothing sets), so both waits run
// out and record ST_TIMEOUT in *status without faulting or hanging the context.
__global__ void wait_probe_kernel(uint32_t* status, const uint32_t* never_set) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait_warp(&bar, 0, &abort_flag, status, 4096);
  // the checkpoint spin of the producer: a bounded poll of a counter that never reaches 1
  bool seen = false;
  for (uint32_t i = 0; i < TC_SYNC_SPIN && !seen; ++i) {
    seen = ld_acquire_u32(never_set) >= 1u;
    __nanosleep(200);
  }
  if (threadIdx.x == 0) {
    if (ok) atomicOr(status, ST_BOUNDS);        // a wait that should not have completed did
    if (!seen) atomicOr(status, ST_TIMEOUT);
  }
}

cudaError_t launch_wait_probe(uint32_t* status, const uint32_t* never_set, cudaStream_t s) {
  count_launch();
  wait_probe_kernel<<<1, 32, 0, s>>>(status, never_set);
  return cudaGetLastError();
}

// ---- host side ---------------------------------------------------------------------------------
// Rows up to 192 wide keep the A tile resident; wider rows stream A and B in K chunks.
constexpr int TC_KRES_MAX = 192;
constexpr int TC_KPAD_MAX = 4096;

bool tc_screen_supported(int d, bool) { return d >= 1 && ((d + 63) / 64) * 64 <= TC_KPAD_MAX; }

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

static bool make_map(CUtensorMap* map, const void* base, int64_t rows, int kpad, int box_rows, bool fp16,
                     std::string* msg) {
  auto enc = get_encode();
  if (!enc) {
    if (msg) *msg = "cuTensorMapEncodeTiled unavailable; ";
    return false;
  }
  cuuint64_t gdim[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_KC, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (msg) *msg = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + "); ";
    return false;
  }
  return true;
}

// 64-bit words for the checkpoint counters (one u32 per checkpoint of the longest producer
// sequence: waves x column tiles).
static size_t sync_counter_words(int64_t m, int64_t n, int grid) {
  const int64_t nrb = (m + TC_BM - 1) / TC_BM;
  const int64_t waves = (nrb + grid - 1) / grid;
  const int64_t ntiles = (n + TC_BN - 1) / TC_BN;
  const int64_t checkpoints = waves * ntiles / TC_SYNC_K + 2;
  return (size_t)((checkpoints + 1) / 2);
}

static uint32_t make_idesc(bool fp16) {
  uint32_t d = 0;
  d |= 1u << 4;                      // D format: F32
  d |= (fp16 ? 0u : 1u) << 7;        // A format: BF16 (1) / F16 (0)
  d |= (fp16 ? 0u : 1u) << 10;       // B format
  // bits 15/16 = 0: A and B K-major
  d |= (uint32_t)(TC_BN >> 3) << 17; // N
  d |= (uint32_t)(128 >> 4) << 24;   // M
  return d;
}

template <int CPL, bool DUMP, bool KSTREAM>
static cudaError_t launch_t(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& p,
                           size_t smem, int grid, cudaStream_t s, float* dump) {
  cudaError_t e = cudaFuncSetAttribute(screen_tc_kernel<CPL, DUMP, KSTREAM>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // cooperative when the producers wait for one another (boundedly): every CTA resident at once
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = p.sync ? 1 : 0;
  count_launch();
  e = cudaLaunchKernelEx(&cfg, screen_tc_kernel<CPL, DUMP, KSTREAM>, ma, mb, p, dump);
  if (e == cudaErrorCooperativeLaunchTooLarge) {  // not all resident: plain launch (waits bounded)
    (void)cudaGetLastError();
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, screen_tc_kernel<CPL, DUMP, KSTREAM>, ma, mb, p, dump);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Pipeline variants the autotuner times: operand stages (0 = as many as shared memory holds,
// else that many fewer), row-buffer capacity step (0 = the smallest that fits, 1 = the next),
// checkpoint lag in windows of 256 tiles.
struct TcVariant {
  int stages_less, cap_step, sync_d;
};
constexpr TcVariant TC_VARIANTS[] = {{0, 0, 8}, {0, 0, 4}, {0, 0, 16}, {1, 0, 8}, {0, 1, 8}, {2, 0, 8}};
constexpr int TC_NVARIANTS = (int)(sizeof(TC_VARIANTS) / sizeof(TC_VARIANTS[0]));

int screen_tc_variants() { return TC_NVARIANTS; }

static cudaError_t launch_impl(const TcScreenArgs& a, cudaStream_t s, std::string* msg, float* dump,
                               int variant, TcShape* shape) {
  if (variant < 0 || variant >= TC_NVARIANTS) {
    if (msg) *msg = "unknown screen variant; ";
    return cudaErrorInvalidValue;
  }
  const TcVariant v = TC_VARIANTS[variant];
  const int kpad = a.kpad;
  if (kpad % 64 != 0 || kpad < 64 || kpad > TC_KPAD_MAX) {
    if (msg) *msg = "kpad must be a multiple of 64 in [64, 4096]; ";
    return cudaErrorInvalidValue;
  }
  const bool kstream = kpad > TC_KRES_MAX;
  TcParams p{};
  p.m = a.m;
  p.n = a.n;
  p.kpad = kpad;
  p.nkc = kpad / 64;
  const int a_bytes = kstream ? 0 : TC_BM * kpad * 2;
  const int stage_bytes = kstream ? (TC_BM + TC_BN) * TC_KC * 2 : TC_BN * kpad * 2;
  const int fixed = 1024 + TC_MAXST * TC_BN * 4 + 256 + 8 * 256 * 4;  // alignment, norms, barriers, hist
  const int budget = 220 * 1024 - a_bytes - fixed;
  p.nst = std::min(TC_MAXST, budget / stage_bytes) - v.stages_less;
  if (p.nst < 2) {
    if (msg) *msg = "shared memory too small for two operand stages; ";
    return cudaErrorInvalidValue;
  }
  p.Lp = a.Lp;
  int cpl = 0, step = v.cap_step;
  for (int c : {12, 16, 20, 24})
    if (c * 32 >= a.Lp + TC_BN + 32 && step-- == 0) { cpl = c; break; }
  if (!cpl) {
    if (msg) *msg = "screened list too long; ";
    return cudaErrorInvalidValue;
  }
  p.cap = cpl * 32;
  p.sync_d = v.sync_d;
  p.row_off = a.row_off;
  if (shape) *shape = TcShape{variant, p.nst, p.cap, p.sync_d};
  p.self_excl = a.self_excl;
  p.idesc = make_idesc(a.fp16);
  p.nb = a.nb;
  p.ids = a.ids;
  p.thr = a.thr;
  p.status = a.status;
  p.perm = dump ? nullptr : a.perm;
  p.wave_start = dump ? 0 : a.wave_start;
  CUtensorMap ma, mb;
  if (!make_map(&ma, a.A, a.m, kpad, TC_BM, a.fp16, msg)) return cudaErrorInvalidValue;
  if (!make_map(&mb, a.B, a.n, kpad, TC_BN, a.fp16, msg)) return cudaErrorInvalidValue;
  const int64_t nrb = (a.m + TC_BM - 1) / TC_BM;
  const int grid = (int)std::min<int64_t>(nrb, num_sms());
  // at least ~116 KB so that a single CTA (and its 512 TMEM columns) fits per SM
  size_t smem = (size_t)fixed + (size_t)a_bytes + (size_t)p.nst * stage_bytes;
  smem = std::max<size_t>(smem, 116 * 1024);
  const size_t buf_words = (size_t)grid * TC_BM * p.cap;
  const size_t sync_words = sync_counter_words(a.m, a.n, grid);
  if (!a.rowbuf || a.rowbuf_words < buf_words + (dump ? 0 : sync_words)) {
    if (msg) *msg = "row buffer missing or too small; ";
    return cudaErrorInvalidValue;
  }
  p.rowbuf = a.rowbuf;
  p.sync = nullptr;
  if (!dump) {  // checkpoint counters after the row buffers, zeroed on the stream
    p.sync = reinterpret_cast<uint32_t*>(a.rowbuf + buf_words);
    cudaError_t ze = cudaMemsetAsync(p.sync, 0, sync_words * 8, s);
    if (ze != cudaSuccess) return ze;
  }
  cudaError_t e;
#define CNG_TC(C)                                                                             \
  case C:                                                                                     \
    if (kstream)                                                                              \
      e = dump ? launch_t<C, true, true>(ma, mb, p, smem, grid, s, dump)                      \
               : launch_t<C, false, true>(ma, mb, p, smem, grid, s, dump);                    \
    else                                                                                      \
      e = dump ? launch_t<C, true, false>(ma, mb, p, smem, grid, s, dump)                     \
               : launch_t<C, false, false>(ma, mb, p, smem, grid, s, dump);                   \
    break;
  switch (cpl) {
    CNG_TC(12)
    CNG_TC(16)
    CNG_TC(20)
    CNG_TC(24)
    default:
      e = cudaErrorInvalidValue;
  }
#undef CNG_TC
  return e;
}

size_t screen_tc_rowbuf_words(int64_t m, int64_t n, int Lp) {
  const int cpl = 24;  // the largest capacity launch_impl may choose
  const int64_t nrb = (m + TC_BM - 1) / TC_BM;
  const int grid = (int)std::min<int64_t>(nrb, num_sms());
  return (size_t)grid * TC_BM * cpl * 32 + sync_counter_words(m, n, grid);
}

// ---- autotuner -----------------------------------------------------------------------------------
// The pipeline variant is chosen once per (device, kpad, L', operand type, self or rows, n
// rounded to a power of two) by timing every valid variant on a sample of two waves of row
// blocks (rows from the middle of the order, their sweep starting where theirs would) against
// all the columns; smaller problems use variant 0.  The results of a screen never depend on
// the variant (the lists are certified and reranked the same way).
struct TunedScreen {
  int dev, kpad, Lp, fp16, self, nlog;
  int variant;
};
static std::mutex g_tc_mu;
static std::vector<TunedScreen> g_tc_tuned;

static int tune_key_nlog(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return l;
}

static cudaError_t tune_variant(const TcScreenArgs& a, cudaStream_t s, std::string* msg, int* chosen) {
  *chosen = 0;
  const int64_t grid = std::min<int64_t>((a.m + TC_BM - 1) / TC_BM, num_sms());
  const int64_t sample = 2 * grid * TC_BM;
  if (a.m < 4 * sample) return cudaSuccess;  // small problems: the default variant
  int dev = 0;
  cudaGetDevice(&dev);
  const TunedScreen key{dev, a.kpad, a.Lp, a.fp16, a.self_excl, tune_key_nlog(a.n), 0};
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    for (const auto& t : g_tc_tuned)
      if (t.dev == key.dev && t.kpad == key.kpad && t.Lp == key.Lp && t.fp16 == key.fp16 &&
          t.self == key.self && t.nlog == key.nlog) {
        *chosen = t.variant;
        return cudaSuccess;
      }
  }
  int32_t* ids = nullptr;
  uint32_t *thr = nullptr, *st = nullptr;
  cudaError_t e = cudaMalloc(&ids, (size_t)sample * a.Lp * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMalloc(&thr, (size_t)sample * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&st, sizeof(uint32_t));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  if (e == cudaSuccess) {
    TcScreenArgs t = a;
    const int64_t off = (a.m / 2 / TC_BM) * TC_BM;
    t.row_off = std::min<int64_t>(off, (a.m - sample) / TC_BM * TC_BM);
    t.A = static_cast<const char*>(a.A) + (size_t)t.row_off * a.kpad * 2;
    t.m = sample;
    t.self_excl = 0;
    t.perm = nullptr;
    t.ids = ids;
    t.thr = thr;
    t.status = st;
    for (int v = 0; v < TC_NVARIANTS && e == cudaSuccess; ++v) {
      for (int rep = 0; rep < (v == 0 ? 2 : 1) && e == cudaSuccess; ++rep) {  // variant 0 warms up
        e = cudaMemsetAsync(st, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) break;
        cudaEventRecord(e0, s);
        std::string m2;
        const cudaError_t le = launch_impl(t, s, &m2, nullptr, v, nullptr);
        cudaEventRecord(e1, s);
        if (le == cudaErrorInvalidValue) {  // variant not valid for this shape
          (void)cudaGetLastError();
          break;
        }
        e = le;
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        uint32_t hst = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost);
        float ms = 0.f;
        if (e == cudaSuccess && hst == 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            (v > 0 || rep == 1) && ms < best) {
          best = ms;
          *chosen = v;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ids);
  cudaFree(thr);
  cudaFree(st);
  if (e != cudaSuccess) {
    if (msg) *msg = "screen autotuning failed; ";
    return e;
  }
  std::lock_guard<std::mutex> lk(g_tc_mu);
  TunedScreen r = key;
  r.variant = *chosen;
  g_tc_tuned.push_back(r);
  return cudaSuccess;
}

cudaError_t launch_screen_tc_tune(const TcScreenArgs& a, cudaStream_t s, std::string* msg, int* variant) {
  return tune_variant(a, s, msg, variant);
}

cudaError_t launch_screen_tc(const TcScreenArgs& a, cudaStream_t s, std::string* msg, TcShape* shape) {
  int variant = a.variant;
  if (variant < 0) {
    cudaError_t e = tune_variant(a, s, msg, &variant);
    if (e != cudaSuccess) return e;
  }
  return launch_impl(a, s, msg, nullptr, variant, shape);
}

cudaError_t launch_screen_tc_dump(const TcScreenArgs& a, float* dump, cudaStream_t s,
                                  std::string* msg) {
  return launch_impl(a, s, msg, dump, 0, nullptr);
}

}  // namespace cng
