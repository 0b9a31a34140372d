// DCT axis passes on the GB300 tensor cores (tcgen05, TMEM accumulators,
// bulk-copy staging), for the grids of a plan with a long axis.
//
// One pass over a grid tensor of shape (pre, n, post) computes, for every
// fibre c = (p, q), y[p, k, q] = sum_j C[k][j] x[p, j, q] (the per-axis DCT of
// Algorithm 3; C is the DCT-I interpolation matrix on the extrema grid or the
// 1/n DCT-II quadrature of Eq. (quad_1D) on the first-kind grid).  As a
// matrix product this is Y = C X with X the n x (pre post) matrix of fibres.
//
// FP64 accuracy from BF16 tensor cores (an error-free splitting in the manner
// of Ozaki's scheme): every row of C and every fibre of X is scaled by a power
// of two below its largest magnitude and rounded to a 56-bit integer, written
// as 8 balanced base-128 digits (digit 0 in [-128, 128], the others in
// [-64, 63]; each exact in BF16).  The product of digit slices s of C and t of
// X is an integer matrix; all products with s + t = g share one scale, and
// their sum over n <= 1024 terms stays below 2^24, so the tensor cores
// accumulate it exactly in FP32 (36 products, 8 accumulators in TMEM).  The
// epilogue combines the 8 exact sums as integers and converts once to FP64:
// the result differs from the exact product by the digits dropped beyond
// s + t = 7, about 2^-56 of sum_j |C[k][j]| |x[j]| per output.
//
// Kernels, per pass:
//   tc_exp_kernel,   the fibres' exponents (one warp per fibre), then their 8
//   tc_digit_kernel  digit slices written as BF16 tiles in the layout the
//                    tensor cores read (K-major, 8 x 16-byte core matrices);
//   tc_gemm_kernel   one CTA of 128 threads per 128 x 64 output tile: warp 0
//                    streams the A and B slices of each K step into shared
//                    memory with bulk copies (4-stage mbarrier pipeline),
//                    one thread of warp 1 issues the 36 tcgen05.mma of the
//                    step, and all four warps read the accumulators back with
//                    tcgen05.ld and write FP64.
// Every wait on an mbarrier is bounded by %globaltimer; on expiry the kernel
// sets the launch's error flag, waits (bounded) for its copies and MMAs,
// frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>

#include "fct_common.cuh"

namespace {

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long timeout_ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 31u) == 0 && globaltimer_ns() - t0 > timeout_ns) return false;
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// whole warp: TMEM allocation of ncols columns, address written to shared memory
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// Shared-memory matrix descriptor: K-major, no swizzle; LBO = byte distance of
// the two core matrices along K, SBO = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of sm_100 and later
  return d;                             // base offset 0, layout type 0 (no swizzle)
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4)                        // D format: F32
                              | (1u << 7)                      // A format: BF16
                              | (1u << 10)                     // B format: BF16
                              | (static_cast<uint32_t>(kTcN >> 3) << 17)   // N >> 3
                              | (static_cast<uint32_t>(kTcM >> 4) << 24);  // M >> 4
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}
// Arrives on the mbarrier once every MMA issued before by this thread is done.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: thread i gets lane (base + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// v * 2^e for an integer e in a wide range (two exact steps when 2^e alone is
// outside the normal range).
__device__ __forceinline__ double scale2(double v, int e) {
  if (e >= -1022 && e <= 1023) return v * __longlong_as_double(static_cast<long long>(e + 1023) << 52);
  const int h = e / 2;
  return (v * __longlong_as_double(static_cast<long long>(h + 1023) << 52)) *
         __longlong_as_double(static_cast<long long>(e - h + 1023) << 52);
}

// (H 2^28 + L) 2^E, correctly rounded to FP64 with integer instructions only
// (GB300's FP64 pipe is narrow; the epilogue converts every output once).
// Exponents outside the normal range take the FP64 route, whose result is
// the same correctly rounded value.
__device__ __forceinline__ double combine_to_double(long long H, long long L, int E) {
  const __int128 v = (static_cast<__int128>(H) << 28) + static_cast<__int128>(L);
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  const unsigned __int128 av = v < 0 ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
  const unsigned long long whi = static_cast<unsigned long long>(av >> 64);
  const unsigned long long wlo = static_cast<unsigned long long>(av);
  int msb = whi ? 127 - __clzll(static_cast<long long>(whi)) : 63 - __clzll(static_cast<long long>(wlo));
  unsigned long long mant;
  const int sh = msb - 52;
  if (sh <= 0) {
    mant = wlo << (-sh);
  } else {
    const unsigned __int128 m = av >> sh;
    const unsigned __int128 rem = av - (m << sh);
    const unsigned __int128 half = static_cast<unsigned __int128>(1) << (sh - 1);
    mant = static_cast<unsigned long long>(m);
    if (rem > half || (rem == half && (mant & 1ull))) {
      mant += 1ull;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        msb += 1;
      }
    }
  }
  const int bexp = msb + E + 1023;  // the value is mant 2^(msb - 52 + E), mant in [2^52, 2^53)
  if (bexp <= 0 || bexp >= 2047)
    return scale2(fma(static_cast<double>(L), 0x1p-28, static_cast<double>(H)), E + 28);
  return __longlong_as_double(static_cast<long long>(sign | (static_cast<unsigned long long>(bexp) << 52) |
                                                     (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ const double* tc_src(int sel, const double* samples, const double* y0, const double* y1) {
  return sel == 0 ? samples : (sel == 1 ? y0 : y1);
}

// ---------------------------------------------------------------------------
// Split, in two kernels per pass:
//   tc_exp_kernel    one warp per fibre: the power of two above the fibre's
//                    largest magnitude (bits of the magnitudes, no FP64 op);
//   tc_digit_kernel  one thread per fibre and 8-element chunk: the 8 digit
//                    slices of x[c][j], written as 16-byte rows of the BF16
//                    tiles (consecutive threads: consecutive fibres).
// Fibres beyond ncols and elements beyond n are zero.
// ---------------------------------------------------------------------------
struct SplitArgs {
  const TcGridPass* gp;
  const int32_t* tasks;  // pairs {gp, ntile}, this pass's first
  const double* samples;
  const double* y0;
  const double* y1;
  unsigned char* b;      // B slices
  int32_t* f;            // column exponents
};

__device__ __forceinline__ int64_t fibre_start(const TcGridPass& g, int c) {
  const int p = c / g.post, q = c - (c / g.post) * g.post;
  return static_cast<int64_t>(p) * g.n * g.post + q;
}

// block = 64 fibres of one N tile x 16 groups of elements: thread (r, gq)
// scans j = gq, gq + 16, ... of fibre r (consecutive threads read
// consecutive fibres, so loads coalesce when the fibres are strided; 8 loads
// in flight per thread); the 16 partial maxima meet in shared memory.
constexpr int kTcExpGroups = 16;
__global__ void __launch_bounds__(kTcN * kTcExpGroups) tc_exp_kernel(const SplitArgs a) {
  __shared__ unsigned long long smax[kTcExpGroups][kTcN];
  const int gi = a.tasks[2 * blockIdx.x], nt = a.tasks[2 * blockIdx.x + 1];
  const TcGridPass g = a.gp[gi];
  const double* x = tc_src(g.in_sel, a.samples, a.y0, a.y1) + g.base;
  const int r = threadIdx.x % kTcN, gq = threadIdx.x / kTcN;
  const int c = nt * kTcN + r;
  unsigned long long mbits = 0;
  if (c < g.ncols) {
    const int64_t c0 = fibre_start(g, c);
#pragma unroll 8
    for (int j = gq; j < g.n; j += kTcExpGroups) {
      const unsigned long long bits =
          static_cast<unsigned long long>(__double_as_longlong(ldcg(x + c0 + static_cast<int64_t>(j) * g.post))) &
          0x7FFFFFFFFFFFFFFFull;
      mbits = bits > mbits ? bits : mbits;
    }
  }
  smax[gq][r] = mbits;
  __syncthreads();
  if (gq == 0) {
#pragma unroll
    for (int q = 1; q < kTcExpGroups; ++q) mbits = smax[q][r] > mbits ? smax[q][r] : mbits;
    int e = 0;
    if (mbits >= 0x7FF0000000000000ull) {
      e = kTcNonFinite;
    } else if (mbits != 0) {
      int bexp = static_cast<int>(mbits >> 52);
      if (bexp == 0) bexp = 1 - (__clzll(static_cast<long long>(mbits)) - 11);  // subnormal maximum
      e = bexp - 1022;  // max < 2^e (the frexp convention)
    }
    a.f[g.f_off + c] = e;
  }
}

// block = 64 fibres x 4 chunks of 8 elements; grid.y walks the chunks
__global__ void __launch_bounds__(256) tc_digit_kernel(const SplitArgs a) {
  const int gi = a.tasks[2 * blockIdx.x], nt = a.tasks[2 * blockIdx.x + 1];
  const TcGridPass g = a.gp[gi];
  const int r = threadIdx.x & (kTcN - 1);
  const int h = blockIdx.y * 4 + (threadIdx.x >> 6);  // 8-element chunk
  if (h >= 2 * g.ksteps) return;
  const int c = nt * kTcN + r;
  const double* x = tc_src(g.in_sel, a.samples, a.y0, a.y1) + g.base;
  const int e = ldcg(a.f + g.f_off + c);
  const bool live = c < g.ncols && e != kTcNonFinite;
  const int64_t c0 = live ? fibre_start(g, c) : 0;
  uint32_t packed[kTcSlices][4];
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    int32_t dg[2][kTcSlices];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = 8 * h + i + u;
      long long v = 0;
      if (live && j < g.n) v = __double2ll_rn(scale2(ldcg(x + c0 + static_cast<int64_t>(j) * g.post), 56 - e));
#pragma unroll
      for (int t = kTcSlices - 1; t >= 1; --t) {
        const long long qd = (v + 64) >> 7;
        dg[u][t] = static_cast<int32_t>(v - qd * 128);
        v = qd;
      }
      dg[u][0] = static_cast<int32_t>(v);
    }
#pragma unroll
    for (int t = 0; t < kTcSlices; ++t) {
      const uint32_t lo = __float_as_uint(static_cast<float>(dg[0][t])) >> 16;
      const uint32_t hi = __float_as_uint(static_cast<float>(dg[1][t])) >> 16;
      packed[t][i / 2] = lo | (hi << 16);
    }
  }
  unsigned char* bt = a.b + g.b_off + (static_cast<int64_t>(nt) * g.ksteps + h / 2) * kTcBStep;
  const int off = (r / 8) * 256 + (h % 2) * 128 + (r % 8) * 16;
#pragma unroll
  for (int t = 0; t < kTcSlices; ++t)
    *reinterpret_cast<uint4*>(bt + t * kTcBTile + off) = make_uint4(packed[t][0], packed[t][1], packed[t][2], packed[t][3]);
}

// ---------------------------------------------------------------------------
// GEMM: one 128 x 64 output tile per CTA (128 threads)
// ---------------------------------------------------------------------------
struct GemmArgs {
  const TcGridPass* gp;
  const int32_t* tasks;   // quads {gp, mtile, ntile, 0}, this pass's first
  const unsigned char* a; // A slices
  const int32_t* a_exp;
  const unsigned char* b; // B slices
  const int32_t* f;
  double* y0;
  double* y1;
  int* err;
  unsigned long long timeout_ns;
};

constexpr int kTcGemmThreads = 128;
constexpr int kTcSmemBytes = kTcStages * kTcStageBytes;
constexpr uint32_t kTcTmemCols = kTcSlices * kTcN;  // 512: one FP32 accumulator per digit sum

__global__ void __launch_bounds__(kTcGemmThreads, 1) tc_gemm_kernel(const GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bars[2 * kTcStages + 1];  // full[s], empty[s], done
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ int s_fexp[kTcN];  // the tile's column exponents
  const int* task = a.tasks + 4 * blockIdx.x;
  const TcGridPass g = a.gp[task[0]];
  const int mt = task[1], nt = task[2];
  const int ksteps = g.ksteps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(&bars[0]);
  auto full = [&](int s) { return bar0 + 8u * static_cast<uint32_t>(s); };
  auto empty = [&](int s) { return bar0 + 8u * static_cast<uint32_t>(kTcStages + s); };
  const uint32_t done = bar0 + 8u * (2 * kTcStages);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), kTcTmemCols);
  if (threadIdx.x < kTcN) {
    const int c = nt * kTcN + static_cast<int>(threadIdx.x);
    s_fexp[threadIdx.x] = c < g.ncols ? ldcg(a.f + g.f_off + c) : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const unsigned char* A = a.a + g.a_off + static_cast<int64_t>(mt) * ksteps * kTcAStep;
  const unsigned char* B = a.b + g.b_off + static_cast<int64_t>(nt) * ksteps * kTcBStep;
  const uint32_t sbase = smem_u32(sm);

  // Warp-specialised roles, each run by a whole warp (the waits are
  // warp-uniform, one elected lane issues): warp 0 streams the A and B slices
  // of every K step into shared memory with bulk copies; warp 1 issues the
  // tensor-core products; warps 2 and 3 wait for the accumulators.
  int issued = 0;  // warp 0: stages whose copies were issued
  if (warp == 0) {
    for (int s = 0; s < ksteps; ++s) {
      const int b = s % kTcStages;
      if (s >= kTcStages) {
        const bool ok = mbar_wait(empty(b), ((s / kTcStages) - 1) & 1, a.timeout_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) atomicExch(&s_fail, 1);
          break;
        }
      }
      if (lane == 0) {
        const uint32_t dst = sbase + static_cast<uint32_t>(b * kTcStageBytes);
        mbar_expect_tx(full(b), kTcStageBytes);
        bulk_g2s(dst, A + static_cast<int64_t>(s) * kTcAStep, kTcAStep, full(b));
        bulk_g2s(dst + kTcAStep, B + static_cast<int64_t>(s) * kTcBStep, kTcBStep, full(b));
      }
      __syncwarp();
      ++issued;
    }
  } else if (warp == 1) {
    // accumulator g (TMEM columns g*64 ..) gathers the products of digit
    // slices s of C and t of X with s + t = g
    for (int s = 0; s < ksteps; ++s) {
      const int b = s % kTcStages;
      const bool ok = mbar_wait(full(b), (s / kTcStages) & 1, a.timeout_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      if (lane == 0) {
        const uint32_t abase = sbase + static_cast<uint32_t>(b * kTcStageBytes);
        const uint32_t bbase = abase + kTcAStep;
#pragma unroll
        for (int grp = 0; grp < kTcSlices; ++grp) {
#pragma unroll
          for (int sa = 0; sa <= grp; ++sa) {
            const uint64_t da = smem_desc(abase + static_cast<uint32_t>(sa * kTcATile), 128, 256);
            const uint64_t db = smem_desc(bbase + static_cast<uint32_t>((grp - sa) * kTcBTile), 128, 256);
            tc_mma(tmem + static_cast<uint32_t>(grp * kTcN), da, db, (s > 0 || sa > 0) ? 1u : 0u);
          }
        }
        tc_commit(empty(b));
      }
      __syncwarp();
    }
    if (lane == 0) tc_commit(done);  // every MMA issued above is complete when `done` flips
    __syncwarp();
  }
  // all threads: wait for the accumulators; the outcome is made uniform over
  // the block (the epilogue's TMEM loads need whole warps)
  if (!mbar_wait(done, 0, a.timeout_ns)) atomicExch(&s_fail, 1);
  tc_fence_after();
  __syncthreads();
  const bool fail = ld_volatile_i32(&s_fail) != 0;
  if (fail) {
    if (threadIdx.x == 0) {  // lane 0 of warp 0, which issued the copies
      atomicCAS(a.err, 0, static_cast<int>(FCT_ERR_TIMEOUT));
      // bounded wait for this CTA's copies still in flight: the last use of
      // every stage buffer
      for (int b = 0; b < kTcStages && b < issued; ++b) {
        const int s_last = b + kTcStages * ((issued - 1 - b) / kTcStages);
        mbar_wait(full(b), (s_last / kTcStages) & 1, a.timeout_ns);
      }
    }
  } else {
    // epilogue: thread (warp w, lane i) owns accumulator row 32 w + i
    const int row = warp * 32 + lane;
    const int k = mt * kTcM + row;
    const bool krow = k < g.n;
    const int ek = krow ? a.a_exp[g.e_off + k] : 0;
    double* out = (g.out_sel == 1 ? a.y0 : a.y1) + g.base;
#pragma unroll 1
    for (int cc = 0; cc < kTcN / 16; ++cc) {
      uint32_t v[kTcSlices][16];
#pragma unroll
      for (int grp = 0; grp < kTcSlices; ++grp)
        tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(grp * kTcN + cc * 16),
                  v[grp]);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = nt * kTcN + cc * 16 + i;
        if (!krow || c >= g.ncols) continue;
        const int fc = s_fexp[cc * 16 + i];
        double y;
        if (fc == kTcNonFinite) {
          y = __longlong_as_double(0x7FF8000000000000ll);
        } else {
          // exact digit sums G_g (integers held in FP32), combined as
          // H = sum_{g<4} G_g 2^(7(3-g)), L = sum_{g>=4} G_g 2^(7(7-g)):
          // y = 2^(e_k + f_c - 35) (H + 2^-28 L)
          // each sum is an integer below 2^27 in magnitude: exact as int32
          long long H = 0, L = 0;
#pragma unroll
          for (int grp = 0; grp < 4; ++grp)
            H = (H << 7) + static_cast<long long>(__float2int_rn(__uint_as_float(v[grp][i])));
#pragma unroll
          for (int grp = 4; grp < kTcSlices; ++grp)
            L = (L << 7) + static_cast<long long>(__float2int_rn(__uint_as_float(v[grp][i])));
          y = combine_to_double(H, L, ek + fc - 63);
        }
        const int p = c / g.post, q = c - (c / g.post) * g.post;
        stcg(out + static_cast<int64_t>(p) * g.n * g.post + static_cast<int64_t>(k) * g.post + q, y);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcTmemCols);
}

fct_status tc_cuda_fail(cudaError_t e, const char* what) {
  (void)cudaGetLastError();
  return fail(FCT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace fct {

TcDevice::~TcDevice() {
  if (mem) cudaFree(mem);
}
TcWork::~TcWork() {
  if (mem) cudaFree(mem);
}

fct_status tc_upload(const TcHost& T, const std::vector<int32_t>& rowbase, const std::vector<int32_t>& rowk,
                     TcDevice* out) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t s_gp = sizeof(TcGridPass) * T.gp.size(), s_split = sizeof(int32_t) * T.split_tasks.size(),
               s_gemm = sizeof(int32_t) * T.gemm_tasks.size(), s_a = sizeof(uint16_t) * T.a_bits.size(),
               s_e = sizeof(int32_t) * T.a_exp.size(), s_po = sizeof(int32_t) * T.pass_chunk_off.size(),
               s_ch = sizeof(DctChunk) * T.dct_chunks.size(), s_gf = sizeof(GridFinal) * T.gfinal.size(),
               s_rb = sizeof(int32_t) * rowbase.size(), s_rk = sizeof(int32_t) * rowk.size();
  const size_t total = al(s_gp) + al(s_split) + al(s_gemm) + al(s_a) + al(s_e) + al(s_po) + al(s_ch) + al(s_gf) +
                       al(s_rb) + al(s_rk);
  char* m = nullptr;
  cudaError_t e = cudaMalloc(&m, total);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(FCT_ERR_OOM, "tensor-core DCT tables")
                                                               : tc_cuda_fail(e, "cudaMalloc(tensor-core DCT tables)");
  out->mem = m;
  size_t off = 0;
  auto put = [&](const void* src, size_t bytes) -> void* {
    void* p = m + off;
    off += al(bytes);
    if (bytes > 0 && e == cudaSuccess) e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
    return p;
  };
  out->gp = static_cast<const TcGridPass*>(put(T.gp.data(), s_gp));
  out->split_tasks = static_cast<const int32_t*>(put(T.split_tasks.data(), s_split));
  out->gemm_tasks = static_cast<const int32_t*>(put(T.gemm_tasks.data(), s_gemm));
  out->a = static_cast<const unsigned char*>(put(T.a_bits.data(), s_a));
  out->a_exp = static_cast<const int32_t*>(put(T.a_exp.data(), s_e));
  out->pass_chunk_off = static_cast<int32_t*>(put(T.pass_chunk_off.data(), s_po));
  out->dct_chunks = static_cast<DctChunk*>(put(T.dct_chunks.data(), s_ch));
  out->gfinal = static_cast<GridFinal*>(put(T.gfinal.data(), s_gf));
  out->rowbase = static_cast<int32_t*>(put(rowbase.data(), s_rb));
  out->rowk = static_cast<int32_t*>(put(rowk.data(), s_rk));
  if (e != cudaSuccess) return tc_cuda_fail(e, "tensor-core DCT upload");
  return FCT_OK;
}

fct_status tc_alloc_work(const TcHost& T, TcWork* out) {
  const size_t sb = (static_cast<size_t>(T.b_bytes) + 255) & ~size_t(255);
  const size_t total = sb + sizeof(int32_t) * static_cast<size_t>(std::max<int64_t>(T.f_count, 1));
  char* m = nullptr;
  cudaError_t e = cudaMalloc(&m, total);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(FCT_ERR_OOM, "tensor-core DCT workspace")
                                                               : tc_cuda_fail(e, "cudaMalloc(tensor-core DCT workspace)");
  out->mem = m;
  out->b = reinterpret_cast<unsigned char*>(m);
  out->f = reinterpret_cast<int32_t*>(m + sb);
  return FCT_OK;
}

fct_status tc_run(const TcHost& T, const TcDevice& D, const TcWork& Wk, const double* samples, double* y0, double* y1,
                  int* err, unsigned long long timeout_ns, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t ea = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
  if (ea != cudaSuccess) return tc_cuda_fail(ea, "tensor-core GEMM shared memory");
  for (int p = 0; p < T.npass; ++p) {
    const int ns = T.split_off[p + 1] - T.split_off[p];
    const int ng = T.gemm_off[p + 1] - T.gemm_off[p];
    if (ns > 0) {
      SplitArgs sa{D.gp, D.split_tasks + 2 * T.split_off[p], samples, y0, y1, Wk.b, Wk.f};
      tc_exp_kernel<<<ns, kTcN * kTcExpGroups, 0, st>>>(sa);
      // chunks of 8 elements: 2 per K step, 4 per block row of the grid
      const unsigned gy = static_cast<unsigned>((2 * T.max_ksteps + 3) / 4);
      tc_digit_kernel<<<dim3(ns, gy), 256, 0, st>>>(sa);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return tc_cuda_fail(e, "tensor-core split launch");
    }
    if (ng > 0) {
      GemmArgs ga{D.gp, D.gemm_tasks + 4 * T.gemm_off[p], D.a, D.a_exp, Wk.b, Wk.f, y0, y1, err, timeout_ns};
      tc_gemm_kernel<<<ng, kTcGemmThreads, kTcSmemBytes, st>>>(ga);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return tc_cuda_fail(e, "tensor-core GEMM launch");
    }
  }
  return FCT_OK;
}

}  // namespace fct
