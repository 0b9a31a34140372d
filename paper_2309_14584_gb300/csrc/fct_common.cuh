// Device helpers shared by the translation units of the GB300 sparse-FCT
// library: global-memory loads and stores, the bounded team barrier, block and
// team reductions, the kernel arguments of the team solver and its template
// declaration (the instantiations live in fct_solve_k<BT>.cu).
#pragma once

#include <cuda_runtime.h>

#include "fct_internal.h"

using namespace fct;

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// Loads of data written earlier in the same launch by other blocks bypass L1
// (ldcg), except the CG gathers of {s, p} and q: those vectors change only in
// the phase before a team barrier, and the barrier's gpu-scope acquire drops
// the SM's L1 lines, so plain loads are current and repeated sectors hit L1.
template <typename T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}
template <typename T>
__device__ __forceinline__ void stcg(T* p, T v) {
  __stcg(p, v);
}

struct Team {
  int G;            // blocks in the team
  int rank;         // this block's rank in the team
  unsigned int epoch;  // barriers passed so far by this block (same in every block)
  TeamBarrier* bar;
  int* err;
  unsigned long long timeout_ns;
};

// Wait (thread 0) until the team counter reaches target, polling with
// gpu-scope acquire loads (measured faster than relaxed polls closed by an
// acq_rel fence).  The error flag and the time limit are checked every 16
// polls, which keeps the poll loop to one load.  Returns 0 when the launch is
// being abandoned (a wait expired here or elsewhere).
__device__ __forceinline__ int bar_wait(const Team& tm, unsigned int target) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned int spin = 1;; ++spin) {
    if (ld_acquire_u32(&tm.bar->count) >= target) return 1;
    if ((spin & 15u) == 0) {
      if (ld_volatile_i32(tm.err) != 0) return 0;
      if (globaltimer_ns() - t0 > tm.timeout_ns) {
        atomicCAS(tm.err, 0, static_cast<int>(FCT_ERR_TIMEOUT));
        return 0;
      }
    }
  }
}

// Team-wide barrier: arrive with a release increment of the team's monotonic
// counter, wait (bounded) until it reaches G x barrier number.  Returns false
// when the launch is being abandoned (a wait expired here or elsewhere).
static __device__ bool team_sync(Team& tm) {
  __shared__ int s_ok;
  __syncthreads();
  tm.epoch += 1;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (tm.G > 1) {
      const unsigned int target = tm.epoch * static_cast<unsigned int>(tm.G);
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&tm.bar->count) : "memory");
      ok = bar_wait(tm, target);
    } else {
      __threadfence();
      if (ld_volatile_i32(tm.err) != 0) ok = 0;
    }
    s_ok = ok;
  }
  __syncthreads();
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// Called once by every block of a team when it leaves the launch: the last
// one out resets the team's counter for the next launch.
static __device__ void team_exit(const Team& tm) {
  __syncthreads();
  if (threadIdx.x == 0 && tm.G > 1) {
    __threadfence();
    const unsigned int n = atomicAdd(&tm.bar->exits, 1u);
    if (n == static_cast<unsigned int>(tm.G - 1)) {
      atomicExch(&tm.bar->count, 0u);
      atomicExch(&tm.bar->exits, 0u);
    }
  }
}

// End of a solver phase: all warps have written their per-warp partials of
// the last nk units (wpart); warp 0 stores the unit partials part[u0 + i*G]
// and its lane 0 arrives at and waits on the team barrier, so one block-wide
// sync before and one after cover both the flush and the barrier.
__device__ __forceinline__ double padd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 padd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double pzero(double) { return 0.0; }
__device__ __forceinline__ double2 pzero(double2) { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------------------
// Sums of squares of FP32 vectors at FP64 accuracy on the FP32 pipe
// (double-float arithmetic): the square of a float is exact as a pair
// hi + lo (hi = v v rounded, lo = fma(v, v, -hi)), and pairs are added with
// Knuth's two-sum, so a warp's sum carries about 48 significant bits.  GB300
// runs FP64 at a small fraction of its FP32 rate, so the FP32 inner solves
// form their inner products this way and convert each warp's pair to FP64
// once per group of units (widen); sums across warps and units are FP64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 df_add(float2 x, float2 y) {
  const float2 s = df_two_sum(x.x, y.x);
  const float e = s.y + (x.y + y.y);
  const float hi = s.x + e;
  return make_float2(hi, e - (hi - s.x));
}
__device__ __forceinline__ float2 df_square(float t) {
  const float hi = t * t;
  return make_float2(hi, fmaf(t, t, -hi));
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
  return v;
}
// Warp sum of values held only by lanes that are multiples of lc (the lead
// lanes of rows or coefficients with lc lanes each; the other lanes hold 0):
// log2(32 / lc) shuffle levels instead of 5, in a fixed order.
__device__ __forceinline__ double warp_sum_from(double v, int lc) {
  for (int o = 16; o >= lc; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum_from(float2 v, int lc) {
  for (int o = 16; o >= lc; o >>= 1)
    v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
  return v;
}
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double widen(float2 v) { return static_cast<double>(v.x) + static_cast<double>(v.y); }

// Per-warp partial of a sum of squares: FP64 for FP64 vectors, a double-float
// pair for FP32 vectors.
template <typename V> struct SqPart;
template <> struct SqPart<double> { using T = double; };
template <> struct SqPart<float> { using T = float2; };
__device__ __forceinline__ double sq_part(double v, double scale) {
  const double t = v * scale;
  return t * t;
}
__device__ __forceinline__ float2 sq_part(float v, double scale) { return df_square(v * static_cast<float>(scale)); }
__device__ __forceinline__ double pzero_part(double) { return 0.0; }
__device__ __forceinline__ float2 pzero_part(float2) { return make_float2(0.0f, 0.0f); }

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return df_add(a, b); }
__device__ __forceinline__ float2 pzero(float2) { return make_float2(0.0f, 0.0f); }

template <int NW, typename PT>
__device__ bool phase_end(Team& tm, const PT (*wpart)[NW], PT* part, int u0, int nk) {
  __shared__ int s_ok2;
  __syncthreads();
  tm.epoch += 1;
  if (threadIdx.x < 32) {
    if (static_cast<int>(threadIdx.x) < nk) {
      PT v = pzero(PT{});
#pragma unroll
      for (int w = 0; w < NW; ++w) v = padd(v, wpart[threadIdx.x][w]);
      stcg(part + u0 + static_cast<int>(threadIdx.x) * tm.G, v);
    }
    __syncwarp();
    if (threadIdx.x == 0) {
      int ok = 1;
      if (tm.G > 1) {
        const unsigned int target = tm.epoch * static_cast<unsigned int>(tm.G);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&tm.bar->count) : "memory");
        ok = bar_wait(tm, target);
      } else {
        __threadfence();
        if (ld_volatile_i32(tm.err) != 0) ok = 0;
      }
      s_ok2 = ok;
    }
    __syncwarp();
  }
  __syncthreads();
  return s_ok2 != 0;
}

// Deterministic block sum; the result is valid in thread 0.
template <int BT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < BT / 32; ++w) r += red[w];
  }
  __syncthreads();
  return r;
}

// Warp 0: sum of n chunk partials in a fixed order (same value in every
// block), left in red[BT/32].
template <int BT>
__device__ __forceinline__ void warp0_team_sum(const double* part, int n, double* red) {
  double v = 0.0;
  for (int i0 = threadIdx.x; i0 < n; i0 += 32 * 8) {
    double t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = ldcg(part + min(i0 + 32 * j, n - 1));  // every load issued
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = i0 + 32 * j < n ? t[j] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) v += t[j];  // lane order: part[lane], part[lane+32], ...
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) red[BT / 32] = v;
}

// Warp 0: FP64 sum of n per-unit partials in a fixed order (lane 0 holds
// the result): 8 independent loads per lane per round, so up to 256
// partials come back in one L2 round trip.
__device__ __forceinline__ double warp0_sum(const double* part, int n) {
  double v = 0.0;
  for (int i0 = threadIdx.x; i0 < n; i0 += 32 * 8) {
    double t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = ldcg(part + min(i0 + 32 * j, n - 1));  // every load issued
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = i0 + 32 * j < n ? t[j] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) v += t[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp 0: double-float sum of n per-unit partials (hi, lo) in a fixed order,
// on the FP32 pipe: 8 independent accumulators per lane (one per load slot of
// a round) keep the dependent chain short; the result (every lane) is the
// pair's FP64 value.
__device__ __forceinline__ double warp0_sum(const float2* part, int n) {
  float2 acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.0f, 0.0f);
  for (int i0 = threadIdx.x; i0 < n; i0 += 32 * 8) {
    float2 t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = ldcg(part + min(i0 + 32 * j, n - 1));  // every load issued
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = i0 + 32 * j < n ? t[j] : make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = df_add(acc[j], t[j]);
  }
  const float2 s = df_add(df_add(df_add(acc[0], acc[1]), df_add(acc[2], acc[3])),
                          df_add(df_add(acc[4], acc[5]), df_add(acc[6], acc[7])));
  return widen(warp_sum(s));
}

// Warp 0: FP64 pair sums of n partials in a fixed order (lane 0 holds the result).
__device__ __forceinline__ double2 warp0_sum(const double2* part, int n) {
  double2 v = make_double2(0.0, 0.0);
  for (int i0 = threadIdx.x; i0 < n; i0 += 32 * 4) {
    double2 t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = ldcg(part + min(i0 + 32 * j, n - 1));  // every load issued
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = i0 + 32 * j < n ? t[j] : make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 4; ++j) v = padd(v, t[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// All threads: team sum of n partials (used outside the overlapped phases).
template <int BT>
__device__ double team_sum(const double* part, int n, double* red) {
  if (threadIdx.x < 32) warp0_team_sum<BT>(part, n, red);
  __syncthreads();
  const double r = red[BT / 32];
  __syncthreads();
  return r;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename V>
__device__ __forceinline__ V lane_group_sum(V v, int L) {
  for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}


template <typename V> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };

struct SolveArgs {
  SolveJob single;          // used when jobs == nullptr
  const SolveJob* jobs;     // device array of njobs jobs, or nullptr
  int njobs;
  int team_blocks;
  LaunchState* ls;
  unsigned long long timeout_ns;
  int smem_bytes;           // dynamic shared memory per block
  ServerRing* ring;         // serving mode when not null (device view of mapped host memory)
  unsigned long long idle_ns;  // serving mode: leave after this long without work
};

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_sys_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_i32(int* p, int v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}


// The team solver kernel (defined in fct_solver.cuh, instantiated per block
// size in fct_solve_k128.cu, fct_solve_k256.cu and fct_solve_k512.cu).
// DEEP = 1: the gathers stage twice as many entries per lane and round (8
// per row lane, 16 per coefficient lane), for plans with long rows or many
// grids, whose gathers stream their tables from DRAM.
template <int BT, bool SV, int DEEP>
__global__ void __launch_bounds__(BT, 512 / BT) fct_solve_kernel(const SolveArgs a);
