// The team solver of the GB300 sparse-FCT library: per-block table staging,
// DCT-I units, alias gathers, CG on the normal equations (FP64, FP32 and the
// pipelined form on A^T A), one transform per team (solve_job) and the
// persistent kernel fct_solve_kernel.  Included only by fct_solve_k<BT>.cu.
#pragma once

#include "fct_common.cuh"

// ---------------------------------------------------------------------------
// Per-block shared-memory copy of the block's static share of the index
// tables.  Every team barrier ends with a gpu-scope acquire, which drops the
// L1 contents, so table reads from global memory would cost an L2 round trip
// at every step of the row -> entry -> column chain; staged in shared memory
// they cost one shared load.  Units beyond the capacity read global memory
// (same arithmetic, same order, same result).
//   A units (rows): header {r0, r1, lanes, jbase, pool offset}; pool holds
//   rowptr[r0..r1] - jbase, then col[jbase .. rowptr[r1]).
//   B units (coefficients): pool holds crow[l][m0 + i] as [K][coefs_per_chunk].
// ---------------------------------------------------------------------------
struct BlockTabs {
  const int* hdrA;      // [nA][5]
  const int* hdrB;      // [nB]
  const int* hdrW;      // [nW][2] {entries, pool offset}
  const int* pool;
  int cachedA, cachedB, cachedW;
  int wbytes;           // entry values staged with the A / B units: 4 (FP32), 8 (FP64) or 0
  const double* mats;   // DCT matrices (shared copy or global)
  void* cmb;            // grid-split A^T q gather: per-warp partials, [2][gather warps][32] doubles
                        // (at the start of the dynamic shared memory), else nullptr
};

// Start (in ints, from the unit's pool offset) of a unit's staged entry
// values: after n index ints, rounded up to 8 bytes.
__device__ __forceinline__ int wt_start(int off, int n) { return (off + n + 1) & ~1; }

//   W units (rows of A^T A, mixed path only; staged first, since the inner
//   solve runs most often): pool holds rowptr[m0..m1] - jbase, the columns,
//   then the FP32 values (as bits).
//   wbytes = 4 / 8: the A and B units also hold the entry values the CG loop
//   reads (FP32 for the mixed path's inner solve, FP64 for the FP64 path),
//   8-byte aligned after the indices.
template <int BT>
__device__ void load_block_tabs(const DevPlan& P, const Team& tm, unsigned char* dsm, int smem_bytes, BlockTabs* T,
                                bool with_w, int wbytes) {
  const int nru = P.n_row_units, ncc = P.n_coef_chunks, nwu = with_w ? P.n_w_units : 0;
  const int nA = nru > tm.rank ? (nru - tm.rank + tm.G - 1) / tm.G : 0;
  const int nB = ncc > tm.rank ? (ncc - tm.rank + tm.G - 1) / tm.G : 0;
  const int nW = nwu > tm.rank ? (nwu - tm.rank + tm.G - 1) / tm.G : 0;
  // grid-split plans: the gather's partial sums first (the host sizes every
  // launch to hold them)
  int off = P.coef_split ? coef_combine_bytes(BT) : 0;
  void* cmb = P.coef_split ? static_cast<void*>(dsm) : nullptr;
  const double* mats = P.dct_mats;
  if (P.mats_smem > 0 && off + static_cast<int>(P.mats_smem * sizeof(double)) <= smem_bytes) {
    double* m = reinterpret_cast<double*>(dsm + off);
    for (int i = threadIdx.x; i < P.mats_smem; i += BT) m[i] = __ldg(P.dct_mats + i);
    mats = m;
    off += P.mats_smem * static_cast<int>(sizeof(double));
  }
  int* hdrA = reinterpret_cast<int*>(dsm + off);
  int* hdrB = hdrA + 5 * nA;
  int* hdrW = hdrB + nB;
  const int nhdr = (5 * nA + nB + 2 * nW + 1) & ~1;  // the pool starts 8-byte aligned
  int* pool = hdrA + nhdr;
  const int cap = (smem_bytes - off) / 4 - nhdr;  // ints left for the pool
  const int wi = wbytes / 4;  // ints per staged entry value
  int used = 0, cachedA = 0, cachedB = 0, cachedW = 0;
  if (cap > 0) {
    for (int k = 0; k < nW; ++k) {
      const int u = tm.rank + k * tm.G;
      const int m0 = u * P.w_rows_per_unit, m1 = min(P.N, m0 + P.w_rows_per_unit);
      const int jbase = __ldg(P.wrowptr + m0), e = __ldg(P.wrowptr + m1) - jbase;
      const int need = (m1 - m0 + 1) + 2 * e;
      if (used + need > cap) break;
      int* rp = pool + used;
      for (int i = threadIdx.x; i <= m1 - m0; i += BT) rp[i] = __ldg(P.wrowptr + m0 + i) - jbase;
      int* cl = rp + (m1 - m0 + 1);
      for (int i = threadIdx.x; i < e; i += BT) {
        cl[i] = __ldg(P.wcol + jbase + i);
        cl[e + i] = __float_as_int(__ldg(P.wval + jbase + i));
      }
      if (threadIdx.x == 0) {
        hdrW[2 * k] = e;
        hdrW[2 * k + 1] = used;
      }
      used += need;
      cachedW = k + 1;
    }
    for (int k = 0; k < nA; ++k) {
      const int u = tm.rank + k * tm.G;
      const int r0 = __ldg(P.ru_first + u), r1 = __ldg(P.ru_first + u + 1);
      const int jbase = __ldg(P.rowptr + r0), jend = __ldg(P.rowptr + r1);
      const int nidx = (r1 - r0 + 1) + (jend - jbase);
      const int need = wi ? wt_start(used, nidx) - used + wi * (jend - jbase) : nidx;
      if (used + need > cap) break;
      int* rp = pool + used;
      for (int i = threadIdx.x; i <= r1 - r0; i += BT) rp[i] = __ldg(P.rowptr + r0 + i) - jbase;
      int* cl = rp + (r1 - r0 + 1);
      for (int i = threadIdx.x; i < jend - jbase; i += BT) cl[i] = __ldg(P.col + jbase + i);
      if (wi == 1) {
        float* wv = reinterpret_cast<float*>(pool + wt_start(used, nidx));
        for (int i = threadIdx.x; i < jend - jbase; i += BT) wv[i] = __ldg(P.wcsr32 + jbase + i);
      } else if (wi == 2) {
        double* wv = reinterpret_cast<double*>(pool + wt_start(used, nidx));
        for (int i = threadIdx.x; i < jend - jbase; i += BT) wv[i] = __ldg(P.wcsr + jbase + i);
      }
      if (threadIdx.x == 0) {
        int* h = hdrA + 5 * k;
        h[0] = r0;
        h[1] = r1;
        h[2] = __ldg(P.ru_lanes + u);
        h[3] = jbase;
        h[4] = used;
      }
      used += need;
      cachedA = k + 1;
    }
    const int cpc = P.coefs_per_chunk;
    const int64_t N = P.N;
    for (int k = 0; k < nB; ++k) {
      const int c = tm.rank + k * tm.G;
      const int nidx = P.K * cpc;
      const int need = wi ? wt_start(used, nidx) - used + wi * nidx : nidx;
      if (used + need > cap) break;
      int* cr = pool + used;
      const int m0 = c * cpc;
      for (int i = threadIdx.x; i < nidx; i += BT) {
        const int l = i / cpc, mm = m0 + i % cpc;
        cr[i] = mm < P.N ? __ldg(P.crow + l * N + mm) : 0;
      }
      if (wi == 1) {
        float* wv = reinterpret_cast<float*>(pool + wt_start(used, nidx));
        for (int i = threadIdx.x; i < nidx; i += BT) {
          const int l = i / cpc, mm = m0 + i % cpc;
          wv[i] = mm < P.N ? __ldg(P.wcm32 + l * N + mm) : 0.0f;
        }
      } else if (wi == 2) {
        double* wv = reinterpret_cast<double*>(pool + wt_start(used, nidx));
        for (int i = threadIdx.x; i < nidx; i += BT) {
          const int l = i / cpc, mm = m0 + i % cpc;
          wv[i] = mm < P.N ? __ldg(P.wcm + l * N + mm) : 0.0;
        }
      }
      if (threadIdx.x == 0) hdrB[k] = used;
      used += need;
      cachedB = k + 1;
    }
  }
  __syncthreads();
  T->hdrA = hdrA;
  T->hdrB = hdrB;
  T->hdrW = hdrW;
  T->pool = pool;
  T->cachedA = cachedA;
  T->cachedB = cachedB;
  T->cachedW = cachedW;
  T->wbytes = wbytes;
  T->mats = mats;
  T->cmb = cmb;
}

// ---------------------------------------------------------------------------
// DCT-I: full axis pass over one work unit (all BT threads)
// ---------------------------------------------------------------------------
// One fibre x[0..N-1] (stride st) of an N-point axis to all N outputs, by the
// symmetry of the DCT matrix: row k satisfies C[k][N-1-j] = (-1)^k C[k][j]
// (DCT-I on extrema points and DCT-II on first-kind points alike), so even
// rows need the pair sums x_j + x_{N-1-j} (plus the middle element when N is
// odd; odd rows vanish there) and odd rows the pair differences: N loads,
// N/2 additions and subtractions, about N^2/2 FMAs.
template <int N>
__device__ __forceinline__ void dct_fibre(const double* C, const double* in, double* out, int st, bool ro) {
  constexpr int H = N / 2;
  double x[N];
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = ro ? __ldg(in + j * st) : ldcg(in + j * st);
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const double a = x[j], b = x[N - 1 - j];
    x[j] = a + b;          // pair sums at 0..H-1
    x[N - 1 - j] = a - b;  // pair differences at N-H..N-1
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const double* Ck = C + k * N;
    double acc = ((N & 1) && !(k & 1)) ? Ck[H] * x[H] : 0.0;
#pragma unroll
    for (int j = 0; j < H; ++j) acc = fma(Ck[j], (k & 1) ? x[N - 1 - j] : x[j], acc);
    stcg(out + k * st, acc);
  }
}

// A work unit of fibres: fibre f = (p, q) of the (pre, n, post = stride) view
// starts at element p n stride + q; consecutive threads take consecutive q.
template <int BT>
__device__ void dct_fibres(const DevPlan& P, const double* mats, const double* __restrict__ samples,
                           const DctChunk& c) {
  double* out = (c.out_sel == 1 ? P.y0 : P.y1) + c.base;
  const double* in = (c.in_sel == 0 ? samples : (c.in_sel == 1 ? P.y0 : P.y1)) + c.base;
  const double* C = mats + c.mat;
  const bool ro = c.in_sel == 0;
  const int st = c.stride;
  for (int f = c.start + static_cast<int>(threadIdx.x); f < c.start + c.count; f += BT) {
    const int p = f / st, q = f - p * st;
    const int64_t b = static_cast<int64_t>(p) * c.n * st + q;
    switch (c.n) {
      case 2: dct_fibre<2>(C, in + b, out + b, st, ro); break;
      case 3: dct_fibre<3>(C, in + b, out + b, st, ro); break;
      case 4: dct_fibre<4>(C, in + b, out + b, st, ro); break;
      case 5: dct_fibre<5>(C, in + b, out + b, st, ro); break;
      case 6: dct_fibre<6>(C, in + b, out + b, st, ro); break;
      case 7: dct_fibre<7>(C, in + b, out + b, st, ro); break;
      case 8: dct_fibre<8>(C, in + b, out + b, st, ro); break;
      case 9: dct_fibre<9>(C, in + b, out + b, st, ro); break;
      case 10: dct_fibre<10>(C, in + b, out + b, st, ro); break;
      case 11: dct_fibre<11>(C, in + b, out + b, st, ro); break;
      case 12: dct_fibre<12>(C, in + b, out + b, st, ro); break;
      case 13: dct_fibre<13>(C, in + b, out + b, st, ro); break;
      case 14: dct_fibre<14>(C, in + b, out + b, st, ro); break;
      case 15: dct_fibre<15>(C, in + b, out + b, st, ro); break;
      default: dct_fibre<16>(C, in + b, out + b, st, ro); break;
    }
  }
}

template <int BT>
__device__ void dct_unit(const DevPlan& P, const double* mats, const double* __restrict__ samples, const DctChunk& c) {
  if (c.fibres) {
    dct_fibres<BT>(P, mats, samples, c);
    return;
  }
  double* out = (c.out_sel == 1 ? P.y0 : P.y1) + c.base;
  const double* C = mats + c.mat;
  const int n = c.n, st = c.stride;
  const double* in = (c.in_sel == 0 ? samples : (c.in_sel == 1 ? P.y0 : P.y1)) + c.base;
  const bool ro = c.in_sel == 0;
  for (int e = c.start + threadIdx.x; e < c.start + c.count; e += BT) {
    const int k = (e / st) % n;
    const int base = e - k * st;
    const double* Ck = C + k * n;
    double acc = 0.0;
    if (ro) {
      for (int j = 0; j < n; ++j) acc = fma(Ck[j], __ldg(in + base + j * st), acc);
    } else {
      for (int j = 0; j < n; ++j) acc = fma(Ck[j], ldcg(in + base + j * st), acc);
    }
    stcg(out + e, acc);
  }
}

// Last pass at a nonempty bin: b[row] = sum_j C[k][j] in[rowbase + j*stride].
// tcm: the tensor-core passes have transformed some grids completely; their
// rows read the result (n = 1) through the kJobTcDct lists.
__device__ __forceinline__ double dct_final_row(const DevPlan& P, const double* mats, const double* __restrict__ samples,
                                                int row, bool tcm) {
  const GridFinal g = (tcm ? P.gfinal_tc : P.gfinal)[__ldg(P.rowgrid + row)];
  const int k = __ldg((tcm ? P.rowk_tc : P.rowk) + row);
  const int base = __ldg((tcm ? P.rowbase_tc : P.rowbase) + row);
  const double* Ck = mats + g.mat + k * g.n;
  double acc = 0.0;
  if (g.in_sel == 0) {
    for (int j = 0; j < g.n; ++j) acc = fma(Ck[j], __ldg(samples + base + j * g.stride), acc);
  } else {
    const double* in = g.in_sel == 1 ? P.y0 : P.y1;
    for (int j = 0; j < g.n; ++j) acc = fma(Ck[j], ldcg(in + base + j * g.stride), acc);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Gather units (worker threads = threads 32..BT-1; warp 0 reduces meanwhile)
//   row unit u: rows ru_first[u] .. ru_first[u+1]-1, ru_lanes[u] lanes per row
//   coef unit c: coefficients c*coefs_per_chunk ..., coef_lanes lanes each
//     (grid-split plans: 32 coefficients, one lane in every gather warp)
// ---------------------------------------------------------------------------
// Row unit geometry: from the block's shared copy (k < cachedA) or global.
struct RowUnit {
  int r0, r1, lc, jbase;
  const int* rp;   // shared rowptr - jbase (nullptr: global)
  const int* cl;   // shared col (relative to jbase)
  const void* wt;  // shared entry values (T.wbytes each, relative to jbase), or nullptr
};

template <bool SV>
__device__ __forceinline__ RowUnit row_unit_geom(const DevPlan& P, const BlockTabs& T, int u, int k) {
  RowUnit g;
  if (k < T.cachedA) {
    const int* h = T.hdrA + 5 * k;
    g.r0 = h[0];
    g.r1 = h[1];
    g.lc = h[2];
    g.jbase = h[3];
    g.rp = T.pool + h[4];
    g.cl = g.rp + (g.r1 - g.r0 + 1);
    if constexpr (SV)
      g.wt = T.wbytes ? static_cast<const void*>(T.pool + wt_start(h[4], (g.r1 - g.r0 + 1) + g.rp[g.r1 - g.r0]))
                      : nullptr;
    else
      g.wt = nullptr;
  } else {
    g.r0 = __ldg(P.ru_first + u);
    g.r1 = __ldg(P.ru_first + u + 1);
    g.lc = __ldg(P.ru_lanes + u);
    g.jbase = 0;
    g.rp = nullptr;
    g.cl = nullptr;
    g.wt = nullptr;
  }
  return g;
}

// Row gather: for each value functor, sum over the row's entries of
// w_j * val(col_j).  Entries are staged EPR per lane at a time (4, or 8 in the
// deep kernel variant for plans with long rows).
template <typename V, typename WT, int NV, bool SV, int EPR, typename Val1, typename Val2>
__device__ __forceinline__ void row_gather_n(const DevPlan& P, const BlockTabs& T, const WT* __restrict__ w, int u,
                                            int k, int wk, int* row_out, bool* lead, Val1 val1, Val2 val2, V* out1,
                                            V* out2) {
  const RowUnit g = row_unit_geom<SV>(P, T, u, k);
  const bool ws = SV && g.wt != nullptr && static_cast<int>(sizeof(WT)) == T.wbytes;
  // a wide unit is one row gathered by every gather thread of the block: each
  // warp returns its partial sum (lead on its lane 0) for wide_row_combine
  const bool wide = g.lc > 32;
  const int gl = wide ? P.workers : g.lc;  // threads on the row
  const int row = wide ? g.r0 : g.r0 + wk / g.lc;
  const int lane = wide ? wk : (wk & (g.lc - 1));
  V a1 = V(0), a2 = V(0);
  if (row < g.r1) {
    int ja, jb;
    if (g.rp) {
      ja = g.rp[row - g.r0];
      jb = g.rp[row - g.r0 + 1];
    } else {
      ja = __ldg(P.rowptr + row);
      jb = __ldg(P.rowptr + row + 1);
    }
    if (g.cl) {
      const int* cl = g.cl;
      const WT* wp = ws ? static_cast<const WT*>(g.wt) : w + g.jbase;
      for (int j0 = ja + lane; j0 < jb; j0 += EPR * gl) {
        int c[EPR];
        WT wv[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) {
          const int j = min(j0 + i * gl, jb - 1);
          c[i] = cl[j];
          wv[i] = ws ? wp[j] : __ldg(wp + j);
        }
        V v[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) v[i] = val1(c[i]);
#pragma unroll
        for (int i = 0; i < EPR; ++i)
          if (j0 + i * gl < jb) a1 = fma(static_cast<V>(wv[i]), v[i], a1);
      }
    } else {
      for (int j0 = ja + lane; j0 < jb; j0 += EPR * gl) {
        int c[EPR];
        WT wv[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) {
          const int j = min(j0 + i * gl, jb - 1);
          c[i] = __ldg(P.col + j);
          wv[i] = __ldg(w + j);
        }
        V v[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) v[i] = val1(c[i]);
#pragma unroll
        for (int i = 0; i < EPR; ++i)
          if (j0 + i * gl < jb) a1 = fma(static_cast<V>(wv[i]), v[i], a1);
      }
    }
  }
  *out1 = lane_group_sum(a1, wide ? 32 : g.lc);
  if (NV > 1) *out2 = lane_group_sum(a2, wide ? 32 : g.lc);
  *row_out = row;
  *lead = (row < g.r1) && (lane & (wide ? 31 : g.lc - 1)) == 0;
}

template <typename V, typename WT, bool SV, int EPR, typename Val>
__device__ __forceinline__ V row_gather(const DevPlan& P, const BlockTabs& T, const WT* __restrict__ w, int u, int k,
                                        int wk, int* row_out, bool* lead, Val val) {
  V a, b;
  row_gather_n<V, WT, 1, SV, EPR>(P, T, w, u, k, wk, row_out, lead, val, val, &a, &b);
  return a;
}

// Phase-A gather of the interleaved {s, p}: as = sum w s[col], ap = sum w p[col]
// (ap skipped on the first iteration, when p is not defined yet).
template <typename V, typename V2, typename WT, bool SV, int EPR>
__device__ __forceinline__ void row_gather_sp(const DevPlan& P, const BlockTabs& T, const WT* __restrict__ w, int u,
                                             int k, int wk, int* row_out, bool* lead, const V2* sp, bool first, V* as,
                                             V* ap) {
  const RowUnit g = row_unit_geom<SV>(P, T, u, k);
  const bool ws = SV && g.wt != nullptr && static_cast<int>(sizeof(WT)) == T.wbytes;
  const bool wide = g.lc > 32;  // see row_gather_n
  const int gl = wide ? P.workers : g.lc;
  const int row = wide ? g.r0 : g.r0 + wk / g.lc;
  const int lane = wide ? wk : (wk & (g.lc - 1));
  V a1 = V(0), a2 = V(0);
  if (row < g.r1) {
    int ja, jb;
    if (g.rp) {
      ja = g.rp[row - g.r0];
      jb = g.rp[row - g.r0 + 1];
    } else {
      ja = __ldg(P.rowptr + row);
      jb = __ldg(P.rowptr + row + 1);
    }
    if (g.cl) {
      const int* cl = g.cl;
      const WT* wp = ws ? static_cast<const WT*>(g.wt) : w + g.jbase;
      for (int j0 = ja + lane; j0 < jb; j0 += EPR * gl) {
        int c[EPR];
        WT wv[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) {
          const int j = min(j0 + i * gl, jb - 1);
          c[i] = cl[j];
          wv[i] = ws ? wp[j] : __ldg(wp + j);
        }
        V2 v[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) v[i] = sp[c[i]];
#pragma unroll
        for (int i = 0; i < EPR; ++i)
          if (j0 + i * gl < jb) {
            a1 = fma(static_cast<V>(wv[i]), v[i].x, a1);
            if (!first) a2 = fma(static_cast<V>(wv[i]), v[i].y, a2);
          }
      }
    } else {
      for (int j0 = ja + lane; j0 < jb; j0 += EPR * gl) {
        int c[EPR];
        WT wv[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) {
          const int j = min(j0 + i * gl, jb - 1);
          c[i] = __ldg(P.col + j);
          wv[i] = __ldg(w + j);
        }
        V2 v[EPR];
#pragma unroll
        for (int i = 0; i < EPR; ++i) v[i] = sp[c[i]];
#pragma unroll
        for (int i = 0; i < EPR; ++i)
          if (j0 + i * gl < jb) {
            a1 = fma(static_cast<V>(wv[i]), v[i].x, a1);
            if (!first) a2 = fma(static_cast<V>(wv[i]), v[i].y, a2);
          }
      }
    }
  }
  *as = lane_group_sum(a1, wide ? 32 : g.lc);
  *ap = lane_group_sum(a2, wide ? 32 : g.lc);
  *row_out = row;
  *lead = (row < g.r1) && (lane & (wide ? 31 : g.lc - 1)) == 0;
}

// Wide rows sort first and are one unit each, so they are the first
// P.n_wide_units row units: a block-uniform test with no memory access.
// A wide unit's warps each hold a partial sum of its row (on the warp's lane
// 0); thread wk = 0 adds them in warp order and becomes the row's only lead.
// Called by every thread of the block (warp 0 included), so the two block
// barriers are reached uniformly.
template <int NGW, typename V>  // NGW = gather warps of the block
__device__ __forceinline__ void wide_row_combine(int wk, V* a, V* b, bool* lead) {
  __shared__ V wsum[2][NGW];
  if (wk >= 0 && (wk & 31) == 0) {
    wsum[0][wk >> 5] = *a;
    wsum[1][wk >> 5] = *b;
  }
  __syncthreads();
  if (wk == 0) {
    V s1 = V(0), s2 = V(0);
    for (int w = 0; w < NGW; ++w) {
      s1 += wsum[0][w];
      s2 += wsum[1][w];
    }
    *a = s1;
    *b = s2;
  }
  *lead = wk == 0;
  __syncthreads();
}

// Coefficient gather: acc = sum over grids l (this lane's share, l = lane,
// lane + L, ...) of w[l][m] * val(crow[l][m]); up to 8 entries per lane are
// staged together.
template <typename V, typename WT, bool SV, int EPC, typename Val>
__device__ __forceinline__ V coef_gather(const DevPlan& P, const BlockTabs& T, const WT* __restrict__ w, int c, int k,
                                         int wk, int* m_out, bool* lead, Val val) {
  // lanes per coefficient and their stride over the grids: L lanes of one
  // warp (lane-split), or lane wk % 32 of every gather warp (grid-split:
  // 32 consecutive coefficients per chunk, warp g takes grids g, g + NW, ...)
  const bool split = P.coef_split != 0;
  const int L = split ? P.workers >> 5 : P.coef_lanes;
  const int cpc = P.coefs_per_chunk;
  const int mi = split ? (wk & 31) : wk / L;
  const int m = c * cpc + mi;
  const int lane = split ? (wk >> 5) : (wk & (L - 1));
  const int* cr = k < T.cachedB ? T.pool + T.hdrB[k] : nullptr;
  const WT* wsm = (SV && cr && static_cast<int>(sizeof(WT)) == T.wbytes)
                      ? reinterpret_cast<const WT*>(T.pool + wt_start(T.hdrB[k], P.K * cpc))
                      : nullptr;
  V acc = V(0);
  if (m < P.N) {
    const int K = P.K;
    const int64_t N = P.N;
    if (cr == nullptr) {
      const int* cg = P.crow + m;
      const WT* wg = w + m;
      for (int lb = lane; lb < K; lb += EPC * L) {
        int idx[EPC];
        WT wv[EPC];
#pragma unroll
        for (int i = 0; i < EPC; ++i) {
          const int64_t l = min(lb + i * L, K - 1);
          idx[i] = __ldg(cg + l * N);
          wv[i] = __ldg(wg + l * N);
        }
        V v[EPC];
#pragma unroll
        for (int i = 0; i < EPC; ++i) v[i] = val(idx[i]);
#pragma unroll
        for (int i = 0; i < EPC; ++i)
          if (lb + i * L < K) acc = fma(static_cast<V>(wv[i]), v[i], acc);
      }
    } else {
      for (int lb = lane; lb < K; lb += EPC * L) {
        int idx[EPC];
        WT wv[EPC];
#pragma unroll
        for (int i = 0; i < EPC; ++i) {
          const int l = min(lb + i * L, K - 1);
          idx[i] = cr[l * cpc + mi];
          wv[i] = wsm ? wsm[l * cpc + mi] : __ldg(w + static_cast<int64_t>(l) * N + m);
        }
        V v[EPC];
#pragma unroll
        for (int i = 0; i < EPC; ++i) v[i] = val(idx[i]);
#pragma unroll
        for (int i = 0; i < EPC; ++i)
          if (lb + i * L < K) acc = fma(static_cast<V>(wv[i]), v[i], acc);
      }
    }
  }
  *m_out = m;
  if (split) {  // the warps' partials are added by coef_combine
    *lead = false;
    return acc;
  }
  acc = lane_group_sum(acc, L);
  *lead = (m < P.N) && lane == 0;
  return acc;
}

// Completes a coefficient gather of chunk number k of this block: in the
// grid-split form, every gather warp's partial goes to shared memory and the
// first gather warp adds them in warp order (lead on its 32 lanes); the
// lane-split form has its sum already.  Called by every thread of the block
// (warp 0 included) once per chunk; the two buffers alternate with k, so one
// block barrier per chunk suffices.
template <int NW, typename V>
__device__ __forceinline__ V coef_combine(const DevPlan& P, const BlockTabs& T, V t, int k, int wk, int m,
                                          bool* lead) {
  if (!P.coef_split) return t;
  V* buf = static_cast<V*>(T.cmb) + (k & 1) * NW * 32;
  if (wk >= 0) buf[wk] = t;
  __syncthreads();
  V s = V(0);
  if (wk >= 0 && wk < 32) {
#pragma unroll
    for (int w = 0; w < NW; ++w) s += buf[w * 32 + wk];
  }
  *lead = wk >= 0 && wk < 32 && m < P.N;
  return s;
}

// The thread that owns coefficient index m of chunk c (updates its vectors).
__device__ __forceinline__ bool coef_owner(const DevPlan& P, int c, int wk, int* m) {
  if (P.coef_split) {
    *m = c * 32 + (wk & 31);
    return wk >= 0 && wk < 32;
  }
  *m = c * P.coefs_per_chunk + wk / P.coef_lanes;
  return (wk & (P.coef_lanes - 1)) == 0;
}

// ---------------------------------------------------------------------------
// Conjugate gradients on the normal equations A^T A x = A^T b, i.e. the CG
// method applied to the least-squares problem of Sec. 3.4 (CGLS in its
// normal-residual form), from x = 0 with s = A^T b, p = s:
//   q = A p;  alpha = |s|^2/|q|^2;  x += alpha p;  s -= alpha A^T q;
//   beta = |s|^2_new / |s|^2;  p = s + beta p.
// One team barrier per matrix product:
//   phase A: q = A s + beta A p from one 16-byte gather of {s, p} per entry,
//            while warp 0 reduces |s|^2 of the previous phase B;
//   phase B: t = A^T q while warp 0 reduces |q|^2; the coefficient owner
//            then writes {s - alpha t, s + beta p} and x + alpha p in place.
// Workers stream through the block's units without block-wide syncs; each
// unit's partial is the fixed-order sum of its warps' sums, so partials (and
// the result) do not depend on the team size.
//
// The inner products that give alpha and beta (|q|^2, |s|^2) are formed at
// FP64 accuracy in a fixed order: FP64 squares and sums for FP64 vectors;
// for FP32 vectors (V = float, the inner solve of the mixed path) exact
// squares summed in double-float arithmetic inside a warp (SqPart), then FP64
// across warps and units.  Squares are taken after scaling by a power of two
// near 1/sqrt(gamma0) (exact), which keeps the FP32 squares of late
// iterations in range.  alpha, beta and the stopping test are computed once
// per block by one thread and broadcast.
// On entry sp[m].x = right-hand side, x = 0, gamma0 = |s|^2 (> 0).  Stops when
// gamma <= tol^2 gamma0, after max_iter (FCT_ERR_NOCONV) or, if stall > 0,
// when gamma has not decreased for `stall` iterations.  All threads of all
// blocks return the same iteration count, final gamma and status.
// ---------------------------------------------------------------------------
constexpr int kUnitGroup = 16;  // units per flush of the per-warp partials


template <int BT, typename V, typename WT, typename XT, bool SV, int DEEP>
__device__ bool cg_normal(const DevPlan& P, Team& tm, const BlockTabs& T, const WT* wcsr, const WT* wcm,
                          typename Vec2<V>::T* sp, V* q, XT* x, double gamma0, double tol, int max_iter, int stall,
                          int* iters_out, double* gamma_out, int* status_out, double* red) {
  using V2 = typename Vec2<V>::T;
  using PT = typename SqPart<V>::T;
  constexpr int NW = BT / 32 - 1;  // worker warps
  __shared__ PT wpart[kUnitGroup][NW];
  __shared__ double sh_ab[2];      // beta, alpha
  __shared__ int sh_ctl[3];        // stop flag, status, iterations
  *status_out = FCT_OK;
  *iters_out = 0;
  *gamma_out = gamma0;
  if (!(gamma0 > 0.0) || !isfinite(gamma0)) {
    if (!isfinite(gamma0)) *status_out = FCT_ERR_NONFINITE;
    return true;
  }
  const int nru = P.n_row_units, ncc = P.n_coef_chunks, nwide = P.n_wide_units;
  const int wk = static_cast<int>(threadIdx.x) - 32;  // worker index; warp 0 has wk < 0
  const int warp = static_cast<int>(threadIdx.x >> 5) - 1;
  const int lane32 = threadIdx.x & 31;
  int e0 = 0;
  frexp(gamma0, &e0);
  const double rs = ldexp(1.0, -(e0 / 2));  // power of two near 1/sqrt(gamma0): exact scaling
  const double c0 = gamma0 * rs * rs;       // gamma0 in scaled units (in [1/4, 4))
  const double tol2 = tol * tol * c0;
  // thread 0's state (scaled gamma)
  double gam = c0, best = c0;
  int it = 0, best_it = 0;
  bool first = true;
  // lead lanes of a unit sit at multiples of its lanes per row (coefficient)
  auto warp_part = [&](int kk, PT v, int lc) {
    v = warp_sum_from(v, lc);
    if (wk >= 0 && lane32 == 0) wpart[kk][warp] = v;
  };
  auto unit_lanes = [&](int u, int k) {
    if (u < nwide) return 32;  // a wide row's sum sits on thread wk = 0 alone
    return k < T.cachedA ? T.hdrA[5 * k + 2] : __ldg(P.ru_lanes + u);
  };
  // per-unit partials: FP64 (FP64 vectors) or double-float pairs (FP32
  // vectors), in the 8-byte slots of part_r / part_c
  PT* const part_r = reinterpret_cast<PT*>(P.part_r);
  PT* const part_c = reinterpret_cast<PT*>(P.part_c);
  auto flush = [&](PT* part, int u0, int nk) {
    __syncthreads();
    if (threadIdx.x < nk) {
      PT v = pzero(PT{});
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) v = padd(v, wpart[threadIdx.x][w2]);
      stcg(part + u0 + threadIdx.x * tm.G, v);
    }
    __syncthreads();
  };
  int ctl = 0;
  for (int pass = 0;; ++pass) {
    // ================= phase A: q = A s + beta A p
    {
      auto gather_a = [&](int u, int k, V* as, V* ap, int* row, bool* lead) {
        row_gather_sp<V, V2, WT, SV, (4 << DEEP)>(P, T, wcsr, u, k, wk, row, lead, sp, first, as, ap);
      };
      int u = tm.rank;
      V as = V(0), ap = V(0);
      int row = 0;
      bool lead = false;
      if (wk >= 0) {
        if (u < nru) gather_a(u, 0, &as, &ap, &row, &lead);
      } else {
        double gnew = 1.0;
        if (!first) gnew = widen(warp0_sum(part_c, ncc));
        if (threadIdx.x == 0) {
          int c = 0;
          double bt = 0.0;
          if (!first) {
            ++it;
            if (!isfinite(gnew)) {
              c = FCT_ERR_NONFINITE + 16;
            } else {
              bt = gnew / gam;
              gam = gnew;
              if (gam <= tol2) c = 1;
              else if (it >= max_iter) c = FCT_ERR_NOCONV + 16;
              else if (stall > 0) {
                if (gam < best) {
                  best = gam;
                  best_it = it;
                } else if (it - best_it >= stall) {
                  c = 1;
                }
              }
            }
          }
          sh_ab[0] = bt;
          sh_ctl[0] = c;
        }
      }
      __syncthreads();
      ctl = sh_ctl[0];
      if (ctl != 0) break;
      const V beta = static_cast<V>(sh_ab[0]);
      int k = 0, kg = 0, u0 = u;
      for (; u < nru; u += tm.G, ++k) {
        if (k > 0 && wk >= 0) gather_a(u, k, &as, &ap, &row, &lead);
        if (u < nwide) wide_row_combine<NW>(wk, &as, &ap, &lead);
        PT part = pzero_part(PT{});
        if (wk >= 0 && lead) {
          const V qv = first ? as : fma(beta, ap, as);
          stcg(q + row, qv);
          part = sq_part(qv, rs);
        }
        warp_part(kg, part, unit_lanes(u, k));
        if (++kg == kUnitGroup && u + tm.G < nru) {
          flush(part_r, u0, kg);
          kg = 0;
          u0 = u + tm.G;
        }
      }
      if (!phase_end<NW>(tm, wpart, part_r, u0, kg)) return false;
    }
    // ================= phase B: t = A^T q; {s, p} and x updated by the owner
    {
      const int L = P.coef_split ? 1 : P.coef_lanes;  // lead lanes sit at multiples of L
      auto own_load = [&](int c, V2* o, XT* xo) {
        int m = 0;
        if (coef_owner(P, c, wk, &m) && m < P.N) {
          *o = ldcg(sp + m);
          *xo = ldcg(x + m);
        }
      };
      int c = tm.rank;
      V t = V(0);
      int m = 0;
      bool lead = false;
      V2 o{};
      XT xo = XT(0);
      if (wk >= 0) {
        if (c < ncc) {
          own_load(c, &o, &xo);
          t = coef_gather<V, WT, SV, (8 << DEEP)>(P, T, wcm, c, 0, wk, &m, &lead, [&](int i) { return q[i]; });
        }
      } else {
        const double dl = widen(warp0_sum(part_r, nru));
        if (threadIdx.x == 0) {
          int cc = 0;
          double al = 0.0;
          if (!isfinite(dl)) cc = FCT_ERR_NONFINITE + 16;
          else if (!(dl > 0.0)) cc = 1;  // q = 0: s is already zero to working precision
          else al = gam / dl;
          sh_ab[1] = al;
          sh_ctl[0] = cc;
          if (P.hist != nullptr && tm.rank == 0 && cc == 0 && pass < P.hist_cap)
            P.hist[pass] = make_double2(al, first ? 0.0 : sh_ab[0]);
        }
      }
      __syncthreads();
      ctl = sh_ctl[0];
      if (ctl != 0) break;
      const V alpha = static_cast<V>(sh_ab[1]);
      const V beta = static_cast<V>(sh_ab[0]);
      int k = 0, kg = 0, c0 = c;
      for (; c < ncc; c += tm.G, ++k) {
        if (k > 0 && wk >= 0) {
          own_load(c, &o, &xo);
          t = coef_gather<V, WT, SV, (8 << DEEP)>(P, T, wcm, c, k, wk, &m, &lead, [&](int i) { return q[i]; });
        }
        t = coef_combine<NW>(P, T, t, k, wk, m, &lead);
        PT part = pzero_part(PT{});
        if (wk >= 0 && lead) {
          const V pn = first ? o.x : fma(beta, o.y, o.x);
          const V sn = fma(-alpha, t, o.x);
          V2 nv;
          nv.x = sn;
          nv.y = pn;
          stcg(sp + m, nv);
          stcg(x + m, static_cast<XT>(fma(static_cast<XT>(alpha), static_cast<XT>(pn), xo)));
          part = sq_part(sn, rs);
        }
        warp_part(kg, part, L);
        if (++kg == kUnitGroup && c + tm.G < ncc) {
          flush(part_c, c0, kg);
          kg = 0;
          c0 = c + tm.G;
        }
      }
      if (!phase_end<NW>(tm, wpart, part_c, c0, kg)) return false;
    }
    first = false;
  }
  // broadcast thread 0's final state
  if (threadIdx.x == 0) {
    sh_ctl[1] = ctl >= 16 ? ctl - 16 : FCT_OK;
    sh_ctl[2] = it;
    sh_ab[0] = gam;
  }
  __syncthreads();
  *status_out = sh_ctl[1];
  *iters_out = sh_ctl[2];
  *gamma_out = sh_ab[0] / (rs * rs);
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Inner solve of the mixed path on the stored normal matrix W = A^T A: CG on
// W d = g in its pipelined form (Ghysels and Vanroose), whose two inner
// products of an iteration are formed together with the vector updates, so
// an iteration is one gather y = W w plus one team barrier (the two-matrix
// form needs a barrier after A p and another after A^T q).
//   vectors (FP32, owned by the thread group of their row): r, p, s = W p,
//   z = W s, w = W r (two buffers: one is gathered while the next is written),
//   x = dx32; right-hand side: sp32[m].x; start x = 0.
//   per iteration, with gamma = r.r, delta = w.r from the previous barrier:
//     beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev)
//     z = y + beta z, s = w + beta s, p = r + beta p
//     x += alpha p, r -= alpha s, w -= alpha z
// The w gathers use plain (L1-cached) loads: every team barrier ends with a
// gpu-scope acquire, which invalidates L1, and w is not written while it is
// gathered.
// ---------------------------------------------------------------------------
template <int BT>
__device__ bool pcg_normal_w(const DevPlan& P, Team& tm, const BlockTabs& T, double gamma0, double tol, int max_iter,
                             int stall, int* iters_out, double* gamma_out, int* status_out) {
  constexpr int NW = BT / 32 - 1;
  __shared__ double2 wpart2[kUnitGroup][NW];
  __shared__ double sh_ab[3];  // alpha, beta, final relative gamma
  __shared__ int sh_ctl[2];    // stop flag, iterations
  *status_out = FCT_OK;
  *iters_out = 0;
  *gamma_out = gamma0;
  if (!(gamma0 > 0.0) || !isfinite(gamma0)) {
    if (!isfinite(gamma0)) *status_out = FCT_ERR_NONFINITE;
    return true;
  }
  const int N = P.N, nwu = P.n_w_units, LW = P.w_lanes, rpw = P.w_rows_per_unit;
  const int wk = static_cast<int>(threadIdx.x) - 32;
  const int warp = static_cast<int>(threadIdx.x >> 5) - 1;
  const int lane32 = threadIdx.x & 31;
  const double rs = 1.0 / sqrt(gamma0);
  const double tol2 = tol * tol;
  float* const wb0 = P.wv;
  float* const wb1 = P.wv + N;
  float* const vr = P.wv + 2 * static_cast<size_t>(N);
  float* const vp = P.wv + 3 * static_cast<size_t>(N);
  float* const vs = P.wv + 4 * static_cast<size_t>(N);
  float* const vz = P.wv + 5 * static_cast<size_t>(N);
  float* const vx = P.dx32;
  const float* const rhs = reinterpret_cast<const float*>(P.sp32);  // .x of {s, p}: stride 2
  // thread 0's state
  double gam_prev = 1.0, al_prev = 1.0, best = 1.0e300, gam_last = 1.0;
  int best_it = 0;

  // y[m] = sum_j W[m][j] src[j * stride] for row m of unit u (k-th unit of this block)
  auto gather = [&](int u, int k, const float* src, int stride, int* m_out, bool* lead) -> float {
    const int g = wk / LW, lane = wk & (LW - 1);
    const int m0 = u * rpw, m = m0 + g;
    *m_out = m;
    *lead = lane == 0 && m < N;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    if (m < N) {
      const int* cl;
      const float* vl;
      int j0, j1;
      if (k < T.cachedW) {
        const int e = T.hdrW[2 * k];
        const int* rp = T.pool + T.hdrW[2 * k + 1];
        const int nrows = min(N, m0 + rpw) - m0;
        cl = rp + nrows + 1;
        vl = reinterpret_cast<const float*>(cl + e);
        j0 = rp[g];
        j1 = rp[g + 1];
      } else {
        cl = P.wcol;
        vl = P.wval;
        j0 = __ldg(P.wrowptr + m);
        j1 = __ldg(P.wrowptr + m + 1);
      }
      int j = j0 + lane;
      for (; j + 3 * LW < j1; j += 4 * LW) {
        const int c0 = cl[j], c1 = cl[j + LW], c2 = cl[j + 2 * LW], c3 = cl[j + 3 * LW];
        const float v0 = vl[j], v1 = vl[j + LW], v2 = vl[j + 2 * LW], v3 = vl[j + 3 * LW];
        a0 = fmaf(v0, src[static_cast<size_t>(c0) * stride], a0);
        a1 = fmaf(v1, src[static_cast<size_t>(c1) * stride], a1);
        a2 = fmaf(v2, src[static_cast<size_t>(c2) * stride], a2);
        a3 = fmaf(v3, src[static_cast<size_t>(c3) * stride], a3);
      }
      for (; j < j1; j += LW) a0 = fmaf(vl[j], src[static_cast<size_t>(cl[j]) * stride], a0);
    }
    return lane_group_sum((a0 + a1) + (a2 + a3), LW);
  };
  auto warp_part2 = [&](int kk, double2 v) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    if (wk >= 0 && lane32 == 0) wpart2[kk][warp] = v;
  };
  auto flush2 = [&](double2* part, int u0, int nk) {
    __syncthreads();
    if (threadIdx.x < nk) {
      double2 v = make_double2(0.0, 0.0);
#pragma unroll
      for (int w2 = 0; w2 < NW; ++w2) v = padd(v, wpart2[threadIdx.x][w2]);
      stcg(part + u0 + threadIdx.x * tm.G, v);
    }
    __syncthreads();
  };

  // ---- set-up: r = g, x = 0, w = W r; partials (r.r, w.r) into buffer 0
  {
    int k = 0, kg = 0, u0 = tm.rank;
    for (int u = tm.rank; u < nwu; u += tm.G, ++k) {
      int m = 0;
      bool lead = false;
      float y = 0.0f;
      if (wk >= 0) y = gather(u, k, rhs, 2, &m, &lead);
      double2 part = make_double2(0.0, 0.0);
      if (wk >= 0 && lead) {
        const float r = ldcg(rhs + 2 * static_cast<size_t>(m));
        stcg(vr + m, r);
        stcg(wb0 + m, y);
        stcg(vx + m, 0.0f);
        const double tr = r * rs, tw = y * rs;
        part = make_double2(tr * tr, tw * tr);
      }
      warp_part2(kg, part);
      if (++kg == kUnitGroup && u + tm.G < nwu) {
        flush2(P.pw64, u0, kg);
        kg = 0;
        u0 = u + tm.G;
      }
    }
    if (!phase_end<NW>(tm, wpart2, P.pw64, u0, kg)) return false;
  }
  int ctl = 0, it = 0;
  for (;; ++it) {
    const float* wcur = (it & 1) ? wb1 : wb0;
    float* wnext = (it & 1) ? wb0 : wb1;
    const double2* pin = P.pw64 + ((it & 1) ? nwu : 0);
    double2* pout = P.pw64 + ((it & 1) ? 0 : nwu);
    int u = tm.rank;
    int m = 0;
    bool lead = false;
    float y = 0.0f, r = 0.0f, pv = 0.0f, sv = 0.0f, zv = 0.0f, xv = 0.0f, wv = 0.0f;
    auto own_load = [&]() {
      r = ldcg(vr + m);
      wv = ldcg(wcur + m);
      xv = ldcg(vx + m);
      if (it > 0) {
        pv = ldcg(vp + m);
        sv = ldcg(vs + m);
        zv = ldcg(vz + m);
      }
    };
    if (wk >= 0) {
      if (u < nwu) {
        y = gather(u, 0, wcur, 1, &m, &lead);
        if (lead) own_load();
      }
    } else {
      const double2 g = warp0_sum(pin, nwu);
      if (threadIdx.x == 0) {
        int c = 0;
        double al = 0.0, bt = 0.0;
        const double gam = g.x, del = g.y;
        gam_last = gam;
        if (!isfinite(gam) || !isfinite(del)) {
          c = FCT_ERR_NONFINITE + 16;
        } else if (gam <= tol2) {
          c = 1;
        } else if (it >= max_iter) {
          c = FCT_ERR_NOCONV + 16;
        } else {
          if (stall > 0) {
            if (gam < best) {
              best = gam;
              best_it = it;
            } else if (it - best_it >= stall) {
              c = 1;
            }
          }
          if (c == 0) {
            bt = it == 0 ? 0.0 : gam / gam_prev;
            const double den = it == 0 ? del : del - bt * gam / al_prev;
            if (!(den > 0.0)) {
              c = 1;  // W is positive semidefinite: no further progress in this precision
            } else {
              al = gam / den;
              gam_prev = gam;
              al_prev = al;
            }
          }
        }
        sh_ab[0] = al;
        sh_ab[1] = bt;
        sh_ctl[0] = c;
      }
    }
    __syncthreads();
    ctl = sh_ctl[0];
    if (ctl != 0) break;
    const float al = static_cast<float>(sh_ab[0]), bt = static_cast<float>(sh_ab[1]);
    int k = 0, kg = 0, u0 = u;
    for (; u < nwu; u += tm.G, ++k) {
      if (k > 0 && wk >= 0) {
        y = gather(u, k, wcur, 1, &m, &lead);
        if (lead) own_load();
      }
      double2 part = make_double2(0.0, 0.0);
      if (wk >= 0 && lead) {
        if (it == 0) {
          zv = y;
          sv = wv;
          pv = r;
        } else {
          zv = fmaf(bt, zv, y);
          sv = fmaf(bt, sv, wv);
          pv = fmaf(bt, pv, r);
        }
        xv = fmaf(al, pv, xv);
        r = fmaf(-al, sv, r);
        wv = fmaf(-al, zv, wv);
        stcg(vz + m, zv);
        stcg(vs + m, sv);
        stcg(vp + m, pv);
        stcg(vx + m, xv);
        stcg(vr + m, r);
        stcg(wnext + m, wv);
        const double tr = r * rs, tw = wv * rs;
        part = make_double2(tr * tr, tw * tr);
      }
      warp_part2(kg, part);
      if (++kg == kUnitGroup && u + tm.G < nwu) {
        flush2(pout, u0, kg);
        kg = 0;
        u0 = u + tm.G;
      }
    }
    if (!phase_end<NW>(tm, wpart2, pout, u0, kg)) return false;
  }
  if (threadIdx.x == 0) {
    sh_ctl[1] = it;
    sh_ab[2] = gam_last;
  }
  __syncthreads();
  *status_out = ctl >= 16 ? ctl - 16 : FCT_OK;
  *iters_out = sh_ctl[1];
  *gamma_out = sh_ab[2] * gamma0;
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// One transform on the team (Algorithm 3): DCT-I of every grid, b at the
// nonempty bins, then the FP64 solve, or FP64 normal-residual sweeps around
// FP32 inner solves (mixed).
// ---------------------------------------------------------------------------
template <int BT, bool SV, int DEEP>
__device__ bool solve_job(const SolveJob& J, Team& tm, double* red, unsigned char* dsm, int smem_bytes) {
  const DevPlan& P = *J.plan;
  if (P.coef_split && smem_bytes < coef_combine_bytes(BT)) {  // the host sizes launches to hold them
    if (threadIdx.x == 0) atomicExch(tm.err, static_cast<int>(FCT_ERR_INVALID_ARG));
    return false;
  }
  BlockTabs T;
  load_block_tabs<BT>(P, tm, dsm, smem_bytes, &T, J.precision == FCT_MIXED && P.n_w_units > 0 && P.s_init == nullptr,
                      SV ? (J.precision == FCT_MIXED ? 4 : 8) : 0);
  const int ncc = P.n_coef_chunks, nre = P.n_rowel_chunks, nru = P.n_row_units, nwide = P.n_wide_units;
  const int wk = static_cast<int>(threadIdx.x) - 32;
  const int nce = (P.N + BT - 1) / BT;  // elementwise units over coefficients
  if (P.s_init != nullptr) {
    // ---- condition probe: x = 0, s = s_init
    for (int u = tm.rank; u < ncc; u += tm.G) {
      const int m = u * BT + threadIdx.x;
      double part = 0.0;
      if (m < P.N) {
        const double v = __ldg(P.s_init + m);
        stcg(P.sp + m, make_double2(v, 0.0));
        stcg(J.coeffs + m, 0.0);
        part = v * v;
      }
      part = block_sum<BT>(part, red);
      if (threadIdx.x == 0) stcg(P.part_c + u, part);
    }
    if (!team_sync(tm)) return false;
  } else {
    // ---- full DCT-I axis passes (kJobTcDct: only the grids left to the FP64
    // units; the tensor-core passes ran before this launch)
    const bool tcm = (J.flags & kJobTcDct) != 0;
    const int npass = tcm ? P.npass_tc : P.npass;
    const int32_t* pco = tcm ? P.pass_chunk_off_tc : P.pass_chunk_off;
    const DctChunk* chunks = tcm ? P.dct_chunks_tc : P.dct_chunks;
    for (int pass = 0; pass < npass; ++pass) {
      const int c0 = __ldg(pco + pass), c1 = __ldg(pco + pass + 1);
      for (int c = c0 + tm.rank; c < c1; c += tm.G) dct_unit<BT>(P, T.mats, J.samples, chunks[c]);
      if (!team_sync(tm)) return false;
    }
    // ---- last pass at the nonempty bins -> b ; x = 0
    for (int u = tm.rank; u < nre + nce; u += tm.G) {
      if (u < nre) {
        const int row = u * BT + threadIdx.x;
        if (row < P.R) stcg(P.b + row, dct_final_row(P, T.mats, J.samples, row, tcm));
      } else {
        const int m = (u - nre) * BT + threadIdx.x;
        if (m < P.N) stcg(J.coeffs + m, 0.0);
      }
    }
    if (!team_sync(tm)) return false;
    // ---- s = A^T b, gamma0 = |A^T b|^2
    for (int c = tm.rank, k = 0; c < ncc; c += tm.G, ++k) {
      int m = 0;
      bool lead = false;
      double t = 0.0;
      if (wk >= 0) t = coef_gather<double, double, SV, (8 << DEEP)>(P, T, P.wcm, c, k, wk, &m, &lead, [&](int i) { return ldcg(P.b + i); });
      t = coef_combine<BT / 32 - 1>(P, T, t, k, wk, m, &lead);
      double part = 0.0;
      if (lead) {
        stcg(P.sp + m, make_double2(t, 0.0));
        part = t * t;
      }
      part = block_sum<BT>(part, red);
      if (threadIdx.x == 0) stcg(P.part_c + c, part);
    }
    if (!team_sync(tm)) return false;
  }
  const double gamma0 = team_sum<BT>(P.part_c, ncc, red);
  if (J.flags & kJobPrepareOnly) return true;  // the DCT stage alone: b and s = A^T b are in place

  int status = FCT_OK, iters = 0, refines = 0;
  double gfinal = gamma0;
  if (!isfinite(gamma0)) {
    status = FCT_ERR_NONFINITE;
  } else if (J.precision != FCT_MIXED) {
    if (!cg_normal<BT, double, double, double, SV, DEEP>(P, tm, T, P.wcsr, P.wcm, P.sp, P.q, J.coeffs, gamma0, J.tol,
                                               J.max_iter, 0, &iters, &gfinal, &status, red))
      return false;
  } else if (gamma0 > 0.0) {
    // Mixed.  g_k = A^T (b - A x_k) in FP64 (g_0 = A^T b); stop when
    // |g_k| <= tol |A^T b|; else solve A^T A d = g_k / |A^T b| in FP32 and
    // set x_{k+1} = x_k + |A^T b| d.
    const double cs = sqrt(gamma0), ci = 1.0 / cs;
    double* x = J.coeffs;
    for (int u = tm.rank; u < nce; u += tm.G) {
      const int m = u * BT + threadIdx.x;
      if (m < P.N) {
        stcg(P.sp32 + m, make_float2(static_cast<float>(ldcg(P.sp + m).x * ci), 0.0f));
        stcg(P.dx32 + m, 0.0f);
      }
    }
    if (!team_sync(tm)) return false;
    double g64 = gamma0;
    for (int k = 0;; ++k) {
      int it_in = 0, st_in = FCT_OK;
      double g_in = 0.0;
      ++refines;
      if (P.n_w_units > 0) {
        if (!pcg_normal_w<BT>(P, tm, T, g64 * ci * ci, J.inner_tol, J.max_iter, 64, &it_in, &g_in, &st_in))
          return false;
      } else if (!cg_normal<BT, float, float, float, SV, DEEP>(P, tm, T, P.wcsr32, P.wcm32, P.sp32, P.q32, P.dx32,
                                                     g64 * ci * ci, J.inner_tol, J.max_iter, 64, &it_in, &g_in,
                                                     &st_in, red)) {
        return false;
      }
      iters += it_in;
      if (st_in == FCT_ERR_NONFINITE) {
        status = st_in;
        break;
      }
      // x += |A^T b| d
      for (int u = tm.rank; u < nce; u += tm.G) {
        const int m = u * BT + threadIdx.x;
        if (m < P.N) stcg(x + m, fma(cs, static_cast<double>(ldcg(P.dx32 + m)), ldcg(x + m)));
      }
      if (!team_sync(tm)) return false;
      // r = b - A x  (FP64)
      for (int u = tm.rank, ku = 0; u < nru; u += tm.G, ++ku) {
        int row = 0;
        bool lead = false;
        double ax = 0.0, unused = 0.0;
        if (wk >= 0)
          ax = row_gather<double, double, SV, (4 << DEEP)>(P, T, P.wcsr, u, ku, wk, &row, &lead,
                                              [&](int m) { return ldcg(x + m); });
        if (u < nwide) wide_row_combine<BT / 32 - 1>(wk, &ax, &unused, &lead);
        if (lead) stcg(P.rres + row, ldcg(P.b + row) - ax);
      }
      if (!team_sync(tm)) return false;
      // g = A^T r (FP64); next inner right-hand side s32 = g / |A^T b|, d = 0
      for (int c = tm.rank, kc = 0; c < ncc; c += tm.G, ++kc) {
        int m = 0;
        bool lead = false;
        double t = 0.0;
        if (wk >= 0)
          t = coef_gather<double, double, SV, (8 << DEEP)>(P, T, P.wcm, c, kc, wk, &m, &lead, [&](int i) { return ldcg(P.rres + i); });
        t = coef_combine<BT / 32 - 1>(P, T, t, kc, wk, m, &lead);
        double part = 0.0;
        if (lead) {
          stcg(P.sp32 + m, make_float2(static_cast<float>(t * ci), 0.0f));
          stcg(P.sp + m, make_double2(t, 0.0));  // for an FP64 continuation
          stcg(P.dx32 + m, 0.0f);
          part = t * t;
        }
        part = block_sum<BT>(part, red);
        if (threadIdx.x == 0) stcg(P.part_c + c, part);
      }
      if (!team_sync(tm)) return false;
      const double g_prev = g64;
      g64 = team_sum<BT>(P.part_c, ncc, red);
      gfinal = g64;
      if (!isfinite(g64)) {
        status = FCT_ERR_NONFINITE;
        break;
      }
      if (!(g64 > 0.0) || g64 <= J.tol * J.tol * gamma0) break;
      if (k + 1 >= J.max_refine || g64 > 1e-2 * g_prev) {
        // FP32 inner solves no longer gain a digit per sweep (an ill-conditioned
        // L-grid): finish in FP64 from the current x, starting from this sweep's
        // exact normal residual g (in sp).
        int it64 = 0, st64 = FCT_OK;
        double g_out = g64;
        const double tol_eff = J.tol * sqrt(gamma0 / g64);
        if (!cg_normal<BT, double, double, double, SV, DEEP>(P, tm, T, P.wcsr, P.wcm, P.sp, P.q, x, g64, tol_eff, J.max_iter,
                                                   0, &it64, &g_out, &st64, red))
          return false;
        iters += it64;
        gfinal = g_out;
        status = st64;
        break;
      }
    }
  }
  if (tm.rank == 0 && threadIdx.x == 0) {
    fct_report rep;
    rep.status = status;
    rep.iterations = iters;
    rep.refinements = refines;
    rep.reserved = 0;
    rep.rel_normal_residual = gamma0 > 0.0 ? sqrt(gfinal / gamma0) : 0.0;
    rep.gamma0 = gamma0;
    *J.report = rep;
  }
  return true;
}

template <int BT, bool SV, int DEEP>
__global__ void __launch_bounds__(BT, 512 / BT) fct_solve_kernel(const SolveArgs a) {
  __shared__ double red[BT / 32 + 2];
  __shared__ int s_job;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int team = blockIdx.x / a.team_blocks;
  Team tm;
  tm.G = a.team_blocks;
  tm.rank = blockIdx.x % a.team_blocks;
  tm.epoch = 0;
  tm.bar = &a.ls->bars[team];
  tm.err = &a.ls->err;
  tm.timeout_ns = a.timeout_ns;
  if (a.ring != nullptr) {
    // Serving: claim published jobs until idle for idle_ns or asked to stop.
    __shared__ SolveJob s_jobdesc;
    for (;;) {
      if (tm.rank == 0 && threadIdx.x == 0) {
        long long got = -1;
        const unsigned long long t0 = globaltimer_ns();
        for (;;) {
          if (ld_acquire_sys_i32(&a.ring->stop) != 0) break;
          if (ld_volatile_i32(&a.ls->exiting) != 0) break;  // the launch is winding down
          if (ld_volatile_i32(&a.ls->err) != 0) break;      // a wait expired somewhere: stop claiming
          const unsigned long long tail = ld_acquire_sys_u64(&a.ring->tail);
          const unsigned int h = ld_volatile_i32(reinterpret_cast<const int*>(&a.ls->queue_head));
          if (h < tail) {
            if (atomicCAS(&a.ls->queue_head, h, h + 1u) == h) {
              got = h;
              atomicAdd(&a.ls->busy, 1);
              break;
            }
            continue;
          }
          // leave only when the whole launch has been idle for idle_ns (no job
          // running, none finished recently): a team that left cannot come
          // back before the next launch
          const unsigned long long now = globaltimer_ns();
          if (now - t0 > a.idle_ns && ld_volatile_i32(&a.ls->busy) == 0 &&
              now - *reinterpret_cast<volatile unsigned long long*>(&a.ls->last_ns) > a.idle_ns) {
            atomicExch(&a.ls->exiting, 1);
            break;
          }
          __nanosleep(256);
        }
        a.ls->team_job[team] = static_cast<int>(got);
      }
      if (!team_sync(tm)) return;
      if (threadIdx.x == 0) {
        const int j = ldcg(&a.ls->team_job[team]);
        s_job = j;
        if (j >= 0) s_jobdesc = a.ring->slots[j % kRingSize].job;
      }
      __syncthreads();
      const int j = s_job;
      const SolveJob J = s_jobdesc;
      __syncthreads();
      if (j < 0) break;
      if (!solve_job<BT, SV, DEEP>(J, tm, red, dsm, a.smem_bytes)) {
        // Abandoned (a bounded wait expired in this team or another one): the
        // job is reported finished with the launch's error code, the error is
        // published in the ring for the host, the job no longer counts as
        // busy, and the launch winds down (the host does not relaunch it).
        if (tm.rank == 0 && threadIdx.x == 0) {
          const int err = ld_volatile_i32(&a.ls->err);
          fct_report rep;
          rep.status = err != 0 ? err : static_cast<int>(FCT_ERR_TIMEOUT);
          rep.iterations = 0;
          rep.refinements = 0;
          rep.reserved = 0;
          rep.rel_normal_residual = 0.0;
          rep.gamma0 = 0.0;
          *J.report = rep;
          st_release_sys_i32(&a.ring->err, rep.status);
          __threadfence_system();
          st_release_sys_i32(&a.ring->slots[j % kRingSize].done, 1);
          atomicExch(&a.ls->exiting, 1);
          __threadfence();
          atomicSub(&a.ls->busy, 1);
        }
        return;
      }
      if (tm.rank == 0 && threadIdx.x == 0) {
        __threadfence_system();
        st_release_sys_i32(&a.ring->slots[j % kRingSize].done, 1);
        atomicExch(&a.ls->last_ns, globaltimer_ns());
        __threadfence();
        atomicSub(&a.ls->busy, 1);
      }
    }
    team_exit(tm);
    return;
  }
  if (a.jobs == nullptr) {
    if (team == 0 && solve_job<BT, SV, DEEP>(a.single, tm, red, dsm, a.smem_bytes)) team_exit(tm);
    return;
  }
  for (;;) {
    if (tm.rank == 0 && threadIdx.x == 0) a.ls->team_job[team] = static_cast<int>(atomicAdd(&a.ls->queue_head, 1u));
    if (!team_sync(tm)) return;
    if (threadIdx.x == 0) s_job = ldcg(&a.ls->team_job[team]);
    __syncthreads();
    const int j = s_job;
    __syncthreads();
    if (j >= a.njobs) break;
    if (!solve_job<BT, SV, DEEP>(a.jobs[j], tm, red, dsm, a.smem_bytes)) return;
  }
  team_exit(tm);
}

