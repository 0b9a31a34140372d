// Device-side construction of a plan's alias tables (the precomputation of
// Sec. 3.3: every column's one entry per grid, Eq. (aliasing_matrix_nd_diff),
// stacked over the L-grid as in Eq. (L-grid_A_mat), empty bins dropped).
//
// The same tables as the host builder, bit for bit:
//   1. fold: one thread per (grid l, coefficient m) walks the nonzero
//      components of m (listed once per coefficient) and computes the global bin
//      key offsets[l] + bin_l(m) and the entry value (signed halves on the
//      first-kind grid, T_m(xi) on single-point axes, multiplied in axis
//      order with round-to-nearest and no contraction, as on the host);
//   2. a stable LSD radix sort of the (key, l N + m) pairs, 8 bits a pass:
//      equal keys keep m ascending, so the sorted order is the bin-sorted
//      CSR of every grid, grids and bins ascending;
//   3. compaction: a row starts where the key changes (flags, exclusive
//      scan) -> rowptr, the row's sample index and grid, columns, values and
//      the coefficient-major row table;
//   4. the device row order: a stable radix sort of the rows, keyed by the
//      gather lane class (most lanes first) and, for 32-lane and wide rows of
//      large plans, the load rounds (most first), then the entries and the
//      row table are permuted to it.
// Everything between the upload of the support and the download of the row
// pointers runs on the device; the host only chooses the entries per lane
// from a 21-counter histogram.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "fct_internal.h"

namespace fct {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // items per block of a radix pass
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // items per block of a scan
constexpr int kElemThreads = 256;

unsigned elem_blocks(int64_t n) {
  const int64_t b = (n + kElemThreads - 1) / kElemThreads;
  return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32)));
}

// T_m(x) by the three-term recurrence, each step rounded as the host's
// t2 = 2 x t1 - t0 (no fused multiply-add).
__device__ double cheb_T_rn(int m, double x) {
  if (m == 0) return 1.0;
  double t0 = 1.0, t1 = x;
  const double x2 = __dmul_rn(2.0, x);
  for (int k = 1; k < m; ++k) {
    const double t2 = __dsub_rn(__dmul_rn(x2, t1), t0);
    t0 = t1;
    t1 = t2;
  }
  return t1;
}

__device__ __forceinline__ int lanes_for_dev(int32_t len, int epl) {
  int lanes = 1;
  while (lanes < 32 && lanes * epl < len) lanes <<= 1;
  if (len > kWideRowFactor * 32 * epl) return kWideLanes;
  return lanes;
}

// 0. nonzero components of every multi-index, in axis order: a zero
// component folds to bin index 0 with entry 1 on every axis kind, so the fold
// visits only the nonzero ones (sparse supports in high D have a few).
// cnt[m] = their number (cnt[N] = 0, so the exclusive scan ends with the total).
__global__ void nz_count_kernel(int64_t N, int D, const uint16_t* __restrict__ support, int32_t* __restrict__ cnt) {
  for (int64_t m = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; m <= N;
       m += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t c = 0;
    if (m < N)
      for (int i = 0; i < D; ++i) c += support[m * D + i] != 0;
    cnt[m] = c;
  }
}

// pairs[nzoff[m] ..] = (axis << 16) | component, axis ascending.
__global__ void nz_fill_kernel(int64_t N, int D, const uint16_t* __restrict__ support,
                               const int32_t* __restrict__ nzoff, uint32_t* __restrict__ pairs) {
  for (int64_t m = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; m < N;
       m += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int32_t o = nzoff[m];
    for (int i = 0; i < D; ++i) {
      const uint32_t c = support[m * D + i];
      if (c != 0) pairs[o++] = (static_cast<uint32_t>(i) << 16) | c;
    }
  }
}

// 1. fold.  e = l N + m (grid-major, so a warp shares one grid's sizes).
__global__ void fold_kernel(int64_t KN, int64_t N, int D, const int32_t* __restrict__ nzoff,
                            const uint32_t* __restrict__ pairs, const int32_t* __restrict__ sizes,
                            const int32_t* __restrict__ strides, const double* __restrict__ nodes,
                            const int64_t* __restrict__ offsets, int first, int32_t* __restrict__ key,
                            int32_t* __restrict__ val, double* __restrict__ weight) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < KN;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t l = e / N, m = e - l * N;
    const int32_t* sz = sizes + l * D;
    const int32_t* st = strides + l * D;
    int64_t bidx = 0;
    double w = 1.0;
    for (int32_t t = nzoff[m], te = nzoff[m + 1]; t < te; ++t) {
      const uint32_t pr = pairs[t];
      const int i = static_cast<int>(pr >> 16);
      const int64_t c = pr & 0xffffu;
      const int64_t n = sz[i];
      if (n >= 2 && first) {
        // aliasing lemma: q = c div 2n, r = c mod 2n
        const int64_t q = c / (2 * n), r = c - q * 2 * n;
        const double sgn = (q & 1) ? -1.0 : 1.0;
        double v;
        int64_t row;
        if (r < n) {
          v = r == 0 ? sgn : 0.5 * sgn;
          row = r;
        } else if (r > n) {
          v = -0.5 * sgn;
          row = 2 * n - r;
        } else {
          v = 0.0;
          row = 0;
        }
        bidx += row * st[i];
        w = __dmul_rn(w, v);
      } else if (n >= 2) {
        const int64_t period = 2 * (n - 1);
        const int64_t r = c % period;
        bidx += (r <= n - 1 ? r : period - r) * st[i];
      } else {
        const double xi = nodes ? nodes[l * D + i] : 1.0;
        w = __dmul_rn(w, cheb_T_rn(static_cast<int>(c), xi));
      }
    }
    key[e] = static_cast<int32_t>(offsets[l] + bidx);
    val[e] = static_cast<int32_t>(e);
    weight[e] = w;
  }
}

// 2. radix pass, histogram: block b counts the digits of items
// [b kSortTile, (b + 1) kSortTile); ghist is digit-major, [256][nblk], so its
// exclusive scan gives every (digit, block) its first output position.
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const int32_t* __restrict__ key, int64_t n,
                                                                  int shift, int32_t* __restrict__ ghist,
                                                                  int64_t nblk) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
  for (int j = threadIdx.x; j < kSortTile; j += kSortThreads) {
    const int64_t i = base + j;
    if (i < n) atomicAdd(&h[(static_cast<uint32_t>(key[i]) >> shift) & 255u], 1);
  }
  __syncthreads();
  ghist[static_cast<int64_t>(threadIdx.x) * nblk + blockIdx.x] = h[threadIdx.x];
}

// 2. radix pass, stable scatter.  Warp w of block b owns the items
// [b kSortTile + w 512, + 512) and ranks them in 16 rounds of 32 consecutive
// items: lanes with equal digits find each other with match.any, the lowest
// of them advances the warp's counter for the digit.  The rank of an item is
// (its digit's start for this block) + (that digit's count in earlier warps)
// + (its rank inside the warp), so equal digits keep their input order.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const int32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n, int shift,
    const int32_t* __restrict__ ghist, int64_t nblk, int32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int32_t cnt[kSortWarps][256];
  __shared__ int32_t gbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < kSortWarps * 256; j += kSortThreads) cnt[j / 256][j % 256] = 0;
  gbase[threadIdx.x] = ghist[static_cast<int64_t>(threadIdx.x) * nblk + blockIdx.x];
  __syncthreads();
  const int64_t wbase = static_cast<int64_t>(blockIdx.x) * kSortTile + warp * (kSortRounds * 32);
  const unsigned lower = (1u << lane) - 1u;
  int32_t k[kSortRounds], v[kSortRounds], loc[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    k[r] = valid ? kin[i] : 0;
    v[r] = valid ? vin[i] : 0;
    const unsigned d = valid ? ((static_cast<uint32_t>(k[r]) >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int32_t before = valid ? cnt[warp][d] : 0;
    __syncwarp();
    if (valid && (peers & lower) == 0) cnt[warp][d] = before + __popc(peers);
    __syncwarp();
    loc[r] = before + __popc(peers & lower);
  }
  __syncthreads();
  {
    // per digit: exclusive prefix of the warps' counts
    const int d = threadIdx.x;
    int32_t run = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      const int32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    if (i < n) {
      const unsigned d = (static_cast<uint32_t>(k[r]) >> shift) & 255u;
      const int64_t pos = static_cast<int64_t>(gbase[d]) + cnt[warp][d] + loc[r];
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
  }
}

// Exclusive scan of 256 per-thread values; *total gets the block's sum.
__device__ int32_t block_exclusive_scan(int32_t x, int32_t* total) {
  __shared__ int32_t wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t s = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < kScanThreads / 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = s;
  }
  __syncthreads();
  const int32_t prefix = (warp > 0 ? wsum[warp - 1] : 0) + inc - x;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return prefix;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int32_t* __restrict__ in, int64_t n,
                                                                   int32_t* __restrict__ partial) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  int32_t s = 0;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    const int64_t i = base + j;
    if (i < n) s += in[i];
  }
  int32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// One block: exclusive scan of the nb block sums in place; total[0] = sum.
__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(int32_t* __restrict__ partial, int64_t nb,
                                                                     int32_t* __restrict__ total) {
  int32_t carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int64_t i = c0 + threadIdx.x;
    const int32_t x = i < nb ? partial[i] : 0;
    int32_t t;
    const int32_t p = block_exclusive_scan(x, &t);
    if (i < nb) partial[i] = carry + p;
    carry += t;
  }
  if (threadIdx.x == 0) total[0] = carry;
}

// out = exclusive scan of in (may be the same buffer): each block reads its
// whole tile before writing any of it.
__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int32_t* in, int64_t n,
                                                                  const int32_t* __restrict__ partial,
                                                                  int32_t* out) {
  __shared__ int32_t s[kScanTile];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    const int64_t i = base + j;
    s[j] = i < n ? in[i] : 0;
  }
  __syncthreads();
  int32_t mine = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) mine += s[threadIdx.x * kScanItems + j];
  int32_t total;
  int32_t run = partial[blockIdx.x] + block_exclusive_scan(mine, &total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int32_t x = s[threadIdx.x * kScanItems + j];
    s[threadIdx.x * kScanItems + j] = run;
    run += x;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < kScanTile; j += kScanThreads) {
    const int64_t i = base + j;
    if (i < n) out[i] = s[j];
  }
}

// 3. compaction.  flag[p] = 1 where a new key (row) starts.
__global__ void row_flag_kernel(const int32_t* __restrict__ skey, int64_t n, int32_t* __restrict__ flag) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x)
    flag[p] = (p == 0 || skey[p] != skey[p - 1]) ? 1 : 0;
}

// excl = exclusive scan of the flags: a row's index is the number of row
// starts before it.
__global__ void csr_fill_kernel(const int32_t* __restrict__ skey, const int32_t* __restrict__ sval,
                                const int32_t* __restrict__ excl, int64_t n, int64_t N,
                                const double* __restrict__ weight, int32_t* __restrict__ rowptr0,
                                int32_t* __restrict__ rowsrc0, int32_t* __restrict__ rowgrid0,
                                int32_t* __restrict__ col0, double* __restrict__ wcsr0, int32_t* __restrict__ crow0) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const bool start = p == 0 || skey[p] != skey[p - 1];
    const int32_t row = excl[p] + (start ? 1 : 0) - 1;
    const int64_t e = sval[p];
    if (start) {
      rowptr0[row] = static_cast<int32_t>(p);
      rowsrc0[row] = skey[p];
      rowgrid0[row] = static_cast<int32_t>(e / N);
    }
    if (p == n - 1) rowptr0[row + 1] = static_cast<int32_t>(n);
    col0[p] = static_cast<int32_t>(e % N);
    wcsr0[p] = weight[e];
    crow0[e] = row;
  }
}

// 4. lane classes.  hist[q][c]: rows whose gather lane count is 2^c (c = 6:
// wide rows) with 2 << q entries per lane (q = 0, 1, 2).
constexpr int kClassCounters = 3 * kLaneClasses;
__global__ void lane_class_kernel(const int32_t* __restrict__ rowptr, int64_t R, int32_t* __restrict__ hist) {
  __shared__ int32_t h[kClassCounters];
  if (threadIdx.x < kClassCounters) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < R;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t len = rowptr[r + 1] - rowptr[r];
#pragma unroll
    for (int q = 0; q < 3; ++q) atomicAdd(&h[q * kLaneClasses + (__ffs(lanes_for_dev(len, 2 << q)) - 1)], 1);
  }
  __syncthreads();
  if (threadIdx.x < kClassCounters) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Row sort key (row_order_key): wide rows first, then 32 lanes, ...; with
// by_rounds, inside the 32-lane and wide classes the rows with more load
// rounds first.
__global__ void row_class_key_kernel(const int32_t* __restrict__ rowptr, int64_t R, int epl, bool by_rounds,
                                     int32_t* __restrict__ key, int32_t* __restrict__ val) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < R;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t len = rowptr[r + 1] - rowptr[r];
    key[r] = row_order_key(len, lanes_for_dev(len, epl), epl, by_rounds);
    val[r] = static_cast<int32_t>(r);
  }
}

// order[nr] = old row of new row nr.  len -> the new row lengths (scanned
// afterwards into the new row pointer).
__global__ void row_perm_kernel(const int32_t* __restrict__ order, int64_t R, const int32_t* __restrict__ rowptr0,
                                const int32_t* __restrict__ rowsrc0, const int32_t* __restrict__ rowgrid0,
                                int32_t* __restrict__ len, int32_t* __restrict__ inv, int32_t* __restrict__ rowsrc,
                                int32_t* __restrict__ rowgrid) {
  for (int64_t nr = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; nr < R;
       nr += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t r = order[nr];
    len[nr] = rowptr0[r + 1] - rowptr0[r];
    inv[r] = static_cast<int32_t>(nr);
    rowsrc[nr] = rowsrc0[r];
    rowgrid[nr] = rowgrid0[r];
  }
}

// Entry p of the new CSR: its row is the last nr with rowptr[nr] <= p (every
// row is nonempty, so rowptr is strictly increasing).
__global__ void entry_perm_kernel(const int32_t* __restrict__ rowptr, int64_t R, const int32_t* __restrict__ order,
                                  const int32_t* __restrict__ rowptr0, const int32_t* __restrict__ col0,
                                  const double* __restrict__ wcsr0, int64_t n, int32_t* __restrict__ col,
                                  double* __restrict__ wcsr, float* __restrict__ wcsr32) {
  for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int64_t lo = 0, hi = R - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (rowptr[mid] <= p) lo = mid;
      else hi = mid - 1;
    }
    const int64_t src = rowptr0[order[lo]] + (p - rowptr[lo]);
    col[p] = col0[src];
    const double w = wcsr0[src];
    wcsr[p] = w;
    wcsr32[p] = __double2float_rn(w);
  }
}

__global__ void coef_table_kernel(const int32_t* __restrict__ crow0, const int32_t* __restrict__ inv,
                                  const double* __restrict__ weight, int64_t n, int32_t* __restrict__ crow,
                                  float* __restrict__ wcm32) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    crow[e] = inv[crow0[e]];
    wcm32[e] = __double2float_rn(weight[e]);
  }
}

// Per row, the start of its fibre in the grid's last DCT pass and its index
// along that fibre (the same integer arithmetic as final_pass_rows).
__global__ void final_rows_kernel(int64_t R, const int32_t* __restrict__ rowsrc, const int32_t* __restrict__ rowgrid,
                                  const int64_t* __restrict__ offsets, const GridFinal* __restrict__ gfinal,
                                  int32_t* __restrict__ rowbase, int32_t* __restrict__ rowk) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < R;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = rowgrid[r];
    const GridFinal g = gfinal[l];
    const int64_t bin = rowsrc[r] - offsets[l];
    const int64_t k = (bin / g.stride) % g.n;
    rowbase[r] = static_cast<int32_t>(offsets[l] + bin - k * g.stride);
    rowk[r] = static_cast<int32_t>(k);
  }
}

__global__ void set_int_kernel(int32_t* dst, int32_t v) { *dst = v; }

fct_status cuda_err(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(FCT_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  return fail(FCT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Exclusive scan of n int32 (in place allowed); the total is left in *total.
void exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* partial, int32_t* total, cudaStream_t st) {
  const int64_t nb = std::max<int64_t>(1, (n + kScanTile - 1) / kScanTile);
  scan_reduce_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, n, partial);
  scan_partials_kernel<<<1, kScanThreads, 0, st>>>(partial, nb, total);
  scan_apply_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, n, partial, out);
}

// Stable LSD radix sort of (key, val) by the low `bits` bits of key (keys are
// non-negative).  The sorted pairs end in (*k, *v); the other pair is scratch.
void radix_sort(int32_t** k, int32_t** v, int32_t** k2, int32_t** v2, int64_t n, int bits, int32_t* ghist,
                int32_t* partial, int32_t* total, cudaStream_t st) {
  const int64_t nblk = (n + kSortTile - 1) / kSortTile;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<static_cast<unsigned>(nblk), kSortThreads, 0, st>>>(*k, n, shift, ghist, nblk);
    exclusive_scan(ghist, ghist, 256 * nblk, partial, total, st);
    radix_scatter_kernel<<<static_cast<unsigned>(nblk), kSortThreads, 0, st>>>(*k, *v, n, shift, ghist, nblk, *k2, *v2);
    std::swap(*k, *k2);
    std::swap(*v, *v2);
  }
}

}  // namespace

void DeviceTables::release() {
  if (mem) {
    // stream-ordered: no device-wide synchronisation, so a plan can be built
    // while other work (a serving launch) runs
    cudaFreeAsync(mem, static_cast<cudaStream_t>(stream));
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  }
  mem = nullptr;
}

fct_status build_device_tables(HostTables* Hp, const uint16_t* support, const int32_t* sizes, const double* nodes,
                               int grid_kind, int workers, int64_t wave, int fixed_epl, int* epl_out,
                               DeviceTables* out, void* stream) {
  HostTables& H = *Hp;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int D = H.D, K = H.K;
  const int64_t N = H.N, KN = static_cast<int64_t>(K) * N;
  out->release();

  // row-major strides of every grid
  std::vector<int32_t> strides(static_cast<size_t>(K) * D);
  for (int l = 0; l < K; ++l) {
    int64_t s = 1;
    for (int i = D - 1; i >= 0; --i) {
      strides[static_cast<size_t>(l) * D + i] = static_cast<int32_t>(s);
      s *= sizes[static_cast<size_t>(l) * D + i];
    }
  }
  const int64_t nblk = (KN + kSortTile - 1) / kSortTile;
  const int64_t scan_max = std::max<int64_t>(KN + 1, 256 * nblk);
  const int64_t nparts = (scan_max + kScanTile - 1) / kScanTile + 1;

  // one scratch allocation
  struct Piece {
    void** dst;
    size_t bytes;
  };
  std::vector<Piece> pieces;
  auto add = [&](void* dst, size_t bytes) { pieces.push_back({reinterpret_cast<void**>(dst), bytes}); };
  uint16_t* d_support;
  int32_t *d_sizes, *d_strides, *d_k0, *d_v0, *d_k1, *d_v1, *d_ghist, *d_part, *d_small;
  int32_t *d_rowptr0, *d_rowsrc0, *d_rowgrid0, *d_col0, *d_crow0, *d_inv, *d_rowsrc, *d_nzoff;
  uint32_t* d_pairs;
  double *d_nodes, *d_weight, *d_wcsr0;
  int64_t* d_offsets;
  GridFinal* d_gfinal;
  add(&d_support, sizeof(uint16_t) * N * D);
  add(&d_nzoff, sizeof(int32_t) * (N + 1));
  add(&d_pairs, sizeof(uint32_t) * N * D);
  add(&d_sizes, sizeof(int32_t) * K * D);
  add(&d_strides, sizeof(int32_t) * K * D);
  add(&d_nodes, sizeof(double) * K * D);
  add(&d_offsets, sizeof(int64_t) * (K + 1));
  add(&d_gfinal, sizeof(GridFinal) * K);
  add(&d_k0, sizeof(int32_t) * KN);
  add(&d_v0, sizeof(int32_t) * KN);
  add(&d_k1, sizeof(int32_t) * KN);
  add(&d_v1, sizeof(int32_t) * KN);
  add(&d_weight, sizeof(double) * KN);
  add(&d_ghist, sizeof(int32_t) * 256 * nblk);
  add(&d_part, sizeof(int32_t) * nparts);
  add(&d_small, sizeof(int32_t) * 32);
  add(&d_rowptr0, sizeof(int32_t) * (KN + 1));
  add(&d_rowsrc0, sizeof(int32_t) * KN);
  add(&d_rowgrid0, sizeof(int32_t) * KN);
  add(&d_col0, sizeof(int32_t) * KN);
  add(&d_wcsr0, sizeof(double) * KN);
  add(&d_crow0, sizeof(int32_t) * KN);
  add(&d_inv, sizeof(int32_t) * KN);
  add(&d_rowsrc, sizeof(int32_t) * KN);
  add(&out->rowptr, sizeof(int32_t) * (KN + 1));
  add(&out->rowgrid, sizeof(int32_t) * KN);
  add(&out->rowbase, sizeof(int32_t) * KN);
  add(&out->rowk, sizeof(int32_t) * KN);
  add(&out->col, sizeof(int32_t) * KN);
  add(&out->wcsr, sizeof(double) * KN);
  add(&out->wcsr32, sizeof(float) * KN);
  add(&out->crow, sizeof(int32_t) * KN);
  add(&out->wcm32, sizeof(float) * KN);
  auto a256 = [](size_t x) { return (std::max<size_t>(x, 1) + 255) & ~size_t(255); };
  size_t total = 0;
  for (auto& pc : pieces) total += a256(pc.bytes);
  void* mem = nullptr;
  cudaError_t e = cudaMallocAsync(&mem, total, st);
  if (e != cudaSuccess) return cuda_err(e, "cudaMallocAsync(device table build)");
  out->mem = mem;
  out->stream = stream;
  {
    size_t off = 0;
    for (auto& pc : pieces) {
      *pc.dst = static_cast<char*>(mem) + off;
      off += a256(pc.bytes);
    }
  }
  out->wcm = d_weight;  // the coefficient-major values are the fold's output

  cudaError_t ue = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (ue == cudaSuccess) ue = x;
  };
  chk(cudaMemcpyAsync(d_support, support, sizeof(uint16_t) * N * D, cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(d_sizes, sizes, sizeof(int32_t) * K * D, cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(d_strides, strides.data(), sizeof(int32_t) * K * D, cudaMemcpyHostToDevice, st));
  if (nodes) chk(cudaMemcpyAsync(d_nodes, nodes, sizeof(double) * K * D, cudaMemcpyHostToDevice, st));
  chk(cudaMemcpyAsync(d_offsets, H.offsets.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st));
  if (static_cast<int>(H.gfinal.size()) != K) {
    out->release();
    return fail(FCT_ERR_INVALID_ARG, "internal: device table build needs the DCT set-up");
  }
  chk(cudaMemcpyAsync(d_gfinal, H.gfinal.data(), sizeof(GridFinal) * K, cudaMemcpyHostToDevice, st));
  if (ue != cudaSuccess) {
    out->release();
    return cuda_err(ue, "device table build upload");
  }

  // 0. nonzero components; 1. fold
  nz_count_kernel<<<elem_blocks(N + 1), kElemThreads, 0, st>>>(N, D, d_support, d_nzoff);
  exclusive_scan(d_nzoff, d_nzoff, N + 1, d_part, d_small, st);
  nz_fill_kernel<<<elem_blocks(N), kElemThreads, 0, st>>>(N, D, d_support, d_nzoff, d_pairs);
  fold_kernel<<<elem_blocks(KN), kElemThreads, 0, st>>>(KN, N, D, d_nzoff, d_pairs, d_sizes, d_strides,
                                                 nodes ? d_nodes : nullptr, d_offsets,
                                                 grid_kind == FCT_GRID_FIRST_KIND ? 1 : 0, d_k0, d_v0, d_weight);
  // 2. stable sort by the global bin key (keys < M)
  int bits = 0;
  while (bits < 31 && ((H.M - 1) >> bits) > 0) ++bits;
  if (bits == 0) bits = 1;
  int32_t *sk = d_k0, *sv = d_v0, *ak = d_k1, *av = d_v1;
  radix_sort(&sk, &sv, &ak, &av, KN, bits, d_ghist, d_part, d_small, st);
  // 3. compaction: flags into ak, scanned in place
  row_flag_kernel<<<elem_blocks(KN), kElemThreads, 0, st>>>(sk, KN, ak);
  exclusive_scan(ak, ak, KN, d_part, d_small, st);
  csr_fill_kernel<<<elem_blocks(KN), kElemThreads, 0, st>>>(sk, sv, ak, KN, N, d_weight, d_rowptr0, d_rowsrc0, d_rowgrid0,
                                                     d_col0, d_wcsr0, d_crow0);
  chk(cudaGetLastError());
  int32_t nflags = 0;  // the flag scan's total: the number of rows
  chk(cudaMemcpyAsync(&nflags, d_small, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  if (ue != cudaSuccess) {
    out->release();
    return cuda_err(ue, "device table build (fold, sort, compaction)");
  }
  const int64_t R = nflags;
  if (R < 1 || R > KN) {
    out->release();
    return fail(FCT_ERR_CUDA, "device table build: row count out of range");
  }

  // entries per lane from the lane-class histogram
  chk(cudaMemsetAsync(d_small, 0, sizeof(int32_t) * 32, st));
  lane_class_kernel<<<elem_blocks(R), kElemThreads, 0, st>>>(d_rowptr0, R, d_small);
  int32_t hist[kClassCounters];
  chk(cudaMemcpyAsync(hist, d_small, sizeof(hist), cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  if (ue != cudaSuccess) {
    out->release();
    return cuda_err(ue, "device table build (lane classes)");
  }
  int64_t classes[3][kLaneClasses];
  for (int q = 0; q < 3; ++q)
    for (int c = 0; c < kLaneClasses; ++c) classes[q][c] = hist[q * kLaneClasses + c];
  const int epl = pick_entries_per_lane(classes, workers, wave, fixed_epl);
  *epl_out = epl;

  // 4. device row order: a stable sort keyed by row_order_key (reuses the
  // sort buffers: the sorted pairs are no longer needed)
  int32_t *rk = d_k0, *rv = d_v0, *rk2 = d_k1, *rv2 = d_v1;
  row_class_key_kernel<<<elem_blocks(R), kElemThreads, 0, st>>>(d_rowptr0, R, epl, KN >= kRoundsOrderMinEntries, rk,
                                                                 rv);
  radix_sort(&rk, &rv, &rk2, &rv2, R, kRowOrderKeyBits, d_ghist, d_part, d_small, st);
  const int32_t* order = rv;
  row_perm_kernel<<<elem_blocks(R), kElemThreads, 0, st>>>(order, R, d_rowptr0, d_rowsrc0, d_rowgrid0, out->rowptr, d_inv,
                                                    d_rowsrc, out->rowgrid);
  exclusive_scan(out->rowptr, out->rowptr, R, d_part, d_small, st);
  set_int_kernel<<<1, 1, 0, st>>>(out->rowptr + R, static_cast<int32_t>(KN));
  entry_perm_kernel<<<elem_blocks(KN), kElemThreads, 0, st>>>(out->rowptr, R, order, d_rowptr0, d_col0, d_wcsr0, KN,
                                                       out->col, out->wcsr, out->wcsr32);
  coef_table_kernel<<<elem_blocks(KN), kElemThreads, 0, st>>>(d_crow0, d_inv, d_weight, KN, out->crow, out->wcm32);
  final_rows_kernel<<<elem_blocks(R), kElemThreads, 0, st>>>(R, d_rowsrc, out->rowgrid, d_offsets, d_gfinal, out->rowbase,
                                                      out->rowk);
  chk(cudaGetLastError());

  H.R = R;
  H.rowptr.assign(R + 1, 0);
  H.rowsrc.assign(R, 0);
  H.rowgrid.clear();  // stays on the device (out->rowgrid)
  chk(cudaMemcpyAsync(H.rowptr.data(), out->rowptr, sizeof(int32_t) * (R + 1), cudaMemcpyDeviceToHost, st));
  chk(cudaMemcpyAsync(H.rowsrc.data(), d_rowsrc, sizeof(int32_t) * R, cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  if (ue != cudaSuccess) {
    out->release();
    return cuda_err(ue, "device table build (row order)");
  }
  if (H.rowptr[R] != KN) {
    out->release();
    return fail(FCT_ERR_CUDA, "device table build: inconsistent row pointer");
  }
  return FCT_OK;
}

fct_status download_device_tables(const DeviceTables& T, HostTables* Hp) {
  const cudaStream_t st = static_cast<cudaStream_t>(T.stream);
  HostTables& H = *Hp;
  const int64_t KN = static_cast<int64_t>(H.K) * H.N;
  H.col.resize(KN);
  H.wcsr.resize(KN);
  H.crow.resize(KN);
  H.weight.resize(KN);
  cudaError_t ue = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (ue == cudaSuccess) ue = x;
  };
  chk(cudaMemcpyAsync(H.col.data(), T.col, sizeof(int32_t) * KN, cudaMemcpyDeviceToHost, st));
  chk(cudaMemcpyAsync(H.wcsr.data(), T.wcsr, sizeof(double) * KN, cudaMemcpyDeviceToHost, st));
  chk(cudaMemcpyAsync(H.crow.data(), T.crow, sizeof(int32_t) * KN, cudaMemcpyDeviceToHost, st));
  chk(cudaMemcpyAsync(H.weight.data(), T.wcm, sizeof(double) * KN, cudaMemcpyDeviceToHost, st));
  chk(cudaStreamSynchronize(st));
  return ue == cudaSuccess ? FCT_OK : cuda_err(ue, "device table download");
}

}  // namespace fct
