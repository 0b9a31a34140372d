// GB300 (sm_103a) device path of the sparse Fast Chebyshev Transform.
//
// One cooperative, persistent kernel runs the whole of Algorithm 3 for one or
// many transforms: the per-grid DCT-I axis passes, the gather of nonempty
// bins into b, and the least-squares solve (CGLS, the "CG method" of Sec. 3.4)
// whose every iteration is one alias gather A p (bin-major, over the
// bin-sorted CSR) and one alias adjoint A^T r (coefficient-major over the
// per-grid row tables), as in the cost model of Sec. 3.5.
//
// Blocks are grouped in teams; a team solves one transform at a time, taken
// from a work queue, and synchronises through a bounded software barrier in
// global memory (every wait has a time limit and reports FCT_ERR_TIMEOUT).
// A CGLS iteration needs two team barriers: the vectors p_new = s + beta p
// and r_new = r - alpha q are formed on the fly inside the gathers from the
// previous buffers (double-buffered), so no barrier is spent on the
// elementwise updates.  All reductions are two-stage with a fixed order
// (per-chunk block sums, then one sum over chunk partials), so a transform's
// result does not depend on the team size or on the rest of the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "fct_common.cuh"

// ---------------------------------------------------------------------------
// Sampler (workload generator, "sample f" of Algorithm 3)
// ---------------------------------------------------------------------------
struct SampleArgs {
  const int32_t* sizes;      // [K*D]
  const int64_t* offsets;    // [K+1]
  const int32_t* node_off;   // [K*D]
  const double* node_pos;
  const double* ttab;        // [node count][dmax+1] T_k at every node (poly families)
  const uint16_t* support;   // [N*D]
  const double* params;
  double* out;
  int64_t M;
  int K, D, N, family, dmax;
};

__global__ void cheb_table_kernel(const double* node_pos, int nnodes, int dmax, double* ttab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nnodes) return;
  const double x = node_pos[j];
  double* t = ttab + static_cast<int64_t>(j) * (dmax + 1);
  double t0 = 1.0, t1 = x;
  t[0] = 1.0;
  if (dmax >= 1) t[1] = x;
  for (int k = 1; k < dmax; ++k) {
    const double t2 = 2.0 * x * t1 - t0;
    t[k + 1] = t2;
    t0 = t1;
    t1 = t2;
  }
}

__global__ void sample_kernel(const SampleArgs a) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= a.M) return;
  int l = 0;
  while (a.offsets[l + 1] <= e) ++l;
  int64_t rem = e - a.offsets[l];
  // axis indices, last axis fastest
  constexpr int kLocalD = 32;
  int idx[kLocalD];
  const bool local = a.D <= kLocalD;
  double q = 0.0, lin = 0.0;
  const double* pa = a.params;
  for (int i = a.D - 1; i >= 0; --i) {
    const int n = a.sizes[l * a.D + i];
    const int j = static_cast<int>(rem % n);
    rem /= n;
    if (local) idx[i] = a.node_off[l * a.D + i] + j;
    const double x = a.node_pos[a.node_off[l * a.D + i] + j];
    if (a.family == FCT_FAMILY_GAUSSCOS || a.family == FCT_FAMILY_POLY_GAUSSCOS) {
      q = fma(pa[i], x * x, q);
      lin = fma(pa[a.D + i], x, lin);
    } else if (a.family == FCT_FAMILY_RATIONAL) {
      q = fma(pa[i], x * x, q);
    }
  }
  double f = 0.0;
  if (a.family == FCT_FAMILY_GAUSSCOS || a.family == FCT_FAMILY_POLY_GAUSSCOS) f = exp(-q) * cos(lin);
  if (a.family == FCT_FAMILY_RATIONAL) f = 1.0 / (1.0 + q);
  if (a.family == FCT_FAMILY_POLY || a.family == FCT_FAMILY_POLY_GAUSSCOS) {
    const double* c = a.family == FCT_FAMILY_POLY ? pa : pa + 2 * a.D;
    const int stride = a.dmax + 1;
    double acc = 0.0;
    for (int m = 0; m < a.N; ++m) {
      const uint16_t* mi = a.support + static_cast<int64_t>(m) * a.D;
      double t = __ldg(c + m);
      for (int i = 0; i < a.D; ++i) {
        int node;
        if (local) {
          node = idx[i];
        } else {
          int64_t r2 = e - a.offsets[l];
          for (int k = a.D - 1; k > i; --k) r2 /= a.sizes[l * a.D + k];
          node = a.node_off[l * a.D + i] + static_cast<int>(r2 % a.sizes[l * a.D + i]);
        }
        t *= __ldg(a.ttab + static_cast<int64_t>(node) * stride + __ldg(mi + i));
      }
      acc += t;
    }
    f += acc;
  }
  a.out[e] = f;
}

// ---------------------------------------------------------------------------
// Polynomial samples through the bins (fast sampler): p restricted to grid l
// is the grid interpolant whose coefficient at bin k is (A^(l) c)_k, so
//   y0 = A c scattered to the full bin tensors, then T_k(x_j) evaluation
// along every active axis gives p at the grid points.  Cost O(KN + M sum n)
// instead of O(M N D) for term-by-term evaluation.
// ---------------------------------------------------------------------------
__global__ void fold_scatter_kernel(const DevPlan* __restrict__ Pp, const double* __restrict__ c) {
  const DevPlan& P = *Pp;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= P.R) return;
  double acc = 0.0;
  const int j1 = P.rowptr[row + 1];
  for (int j = P.rowptr[row]; j < j1; ++j) acc = fma(P.wcsr[j], c[P.col[j]], acc);
  const GridFinal g = P.gfinal[P.rowgrid[row]];
  P.y0[P.rowbase[row] + static_cast<int64_t>(P.rowk[row]) * g.stride] = acc;
}

__global__ void eval_pass_kernel(const DevPlan* __restrict__ Pp, const DctChunk* __restrict__ chunks, int c0,
                                 const double* __restrict__ mats, double* samples, int add) {
  const DevPlan& P = *Pp;
  const DctChunk ch = chunks[c0 + blockIdx.x];
  const double* in = (ch.in_sel == 1 ? P.y0 : P.y1) + ch.base;
  double* out = (ch.out_sel == 3 ? samples : (ch.out_sel == 1 ? P.y0 : P.y1)) + ch.base;
  const double* E = mats + ch.mat;
  for (int e = ch.start + threadIdx.x; e < ch.start + ch.count; e += blockDim.x) {
    const int j = (e / ch.stride) % ch.n;  // output node index on this axis
    const int base = e - j * ch.stride;
    const double* Ej = E + j * ch.n;
    double acc = 0.0;
    for (int k = 0; k < ch.n; ++k) acc = fma(Ej[k], in[base + k * ch.stride], acc);
    if (ch.out_sel == 3 && add) acc += out[e];
    out[e] = acc;
  }
}

// ---------------------------------------------------------------------------
// The alias operator on its own (fct_plan_apply): y = A x over the bin-major
// CSR (one thread per row, entries in CSR order) and x = A^T y over the
// coefficient-major table (one thread per coefficient, grids in order), the
// same tables and FP64 entries the solver uses.
// ---------------------------------------------------------------------------
__global__ void alias_apply_kernel(const DevPlan* __restrict__ Pp, const double* __restrict__ in,
                                   double* __restrict__ out, int transpose) {
  const DevPlan& P = *Pp;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (!transpose) {
    if (i >= P.R) return;
    double acc = 0.0;
    for (int j = P.rowptr[i]; j < P.rowptr[i + 1]; ++j) acc = fma(P.wcsr[j], in[P.col[j]], acc);
    out[i] = acc;
  } else {
    if (i >= P.N) return;
    double acc = 0.0;
    for (int l = 0; l < P.K; ++l) {
      const int64_t e = static_cast<int64_t>(l) * P.N + i;
      acc = fma(P.wcm[e], in[P.crow[e]], acc);
    }
    out[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// Evaluation of the expansion p(x) = sum_m c_m prod_i T_{m_i}(x_i) at
// arbitrary points (how the paper measures approximation error).  One warp
// per point: its lanes build the point's T_k(x_i) tables (three-term
// recurrence, k <= dmax) in shared memory; the block then streams the support
// and coefficients through shared memory in tiles of kEvalTile terms, and each
// warp sums its point's terms lane-strided and reduces by shuffles (a fixed
// order).
// ---------------------------------------------------------------------------
constexpr int kEvalTile = 256;

__global__ void eval_expansion_kernel(const uint16_t* __restrict__ support, const double* __restrict__ coeffs,
                                      int N, int D, int dmax, const double* __restrict__ points, int64_t P,
                                      double* __restrict__ values) {
  extern __shared__ __align__(16) unsigned char esm[];
  const int ppb = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tk = dmax + 1;
  double* ctile = reinterpret_cast<double*>(esm);                              // [kEvalTile]
  double* tab = ctile + kEvalTile + static_cast<size_t>(warp) * D * tk;        // [D][dmax+1] of this warp
  uint16_t* stile = reinterpret_cast<uint16_t*>(ctile + kEvalTile + static_cast<size_t>(ppb) * D * tk);
  const int64_t p = static_cast<int64_t>(blockIdx.x) * ppb + warp;
  if (p < P) {
    for (int i = lane; i < D; i += 32) {
      const double x = points[p * D + i];
      double* t = tab + static_cast<size_t>(i) * tk;
      double t0 = 1.0, t1 = x;
      t[0] = 1.0;
      if (dmax >= 1) t[1] = x;
      for (int k = 2; k <= dmax; ++k) {
        const double t2 = 2.0 * x * t1 - t0;
        t[k] = t2;
        t0 = t1;
        t1 = t2;
      }
    }
  }
  double acc = 0.0;
  for (int m0 = 0; m0 < N; m0 += kEvalTile) {
    const int nt = min(kEvalTile, N - m0);
    __syncthreads();
    for (int j = threadIdx.x; j < nt; j += blockDim.x) ctile[j] = coeffs[m0 + j];
    for (int e = threadIdx.x; e < nt * D; e += blockDim.x) stile[e] = support[static_cast<size_t>(m0) * D + e];
    __syncthreads();
    if (p < P) {
      for (int j = lane; j < nt; j += 32) {
        double term = ctile[j];
        const uint16_t* mj = stile + static_cast<size_t>(j) * D;
        for (int i = 0; i < D; ++i) term *= tab[static_cast<size_t>(i) * tk + mj[i]];
        acc += term;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (p < P && lane == 0) values[p] = acc;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct fct_plan_s {
  int device = 0;
  fct_options opt{};
  HostTables H;
  int D = 0, K = 0;
  int64_t N = 0, M = 0, R = 0;
  int dmax = 0;
  std::vector<int32_t> sizes;
  // device memory
  char* dmem = nullptr;
  size_t dbytes = 0;
  std::shared_ptr<char> tables;  // owns dmem of the plan that built the tables (shared by clones)
  char* wmem = nullptr;          // a clone's own workspace allocation
  DevPlan hp{};
  DevPlan* dp = nullptr;
  LaunchState* ls = nullptr;
  fct_report* drep = nullptr;
  SolveJob* djobs = nullptr;     // batch job array (grown on demand)
  char* d_hist_block = nullptr;  // condition estimate: DevPlan copy + coefficient history
  int hist_cap = 0;
  int djobs_cap = 0;
  // sampler
  int32_t* d_sizes = nullptr;
  int64_t* d_offsets = nullptr;
  int32_t* d_node_off = nullptr;
  double* d_node_pos = nullptr;
  uint16_t* d_support = nullptr;
  double* d_ttab = nullptr;
  DctChunk* d_ichunks = nullptr;   // evaluation passes of the fast sampler
  double* d_emats = nullptr;
  double* d_params = nullptr;
  int64_t params_cap = 0;
  // host-buffer execute staging
  double* d_stage_in = nullptr;
  double* d_stage_out = nullptr;
  // launch shape
  int block_threads = 256;
  int grid_blocks = 0;
  int max_coresident = 0;
  int blocks_per_sm = 1;
  int smem_bytes = 0;          // dynamic shared memory requested per block
  int smem_cap = 0;            // largest request that keeps blocks_per_sm resident
  std::vector<int32_t> ru_first, rowptr_h;  // for the shared-memory sizing of other team sizes
  std::vector<int32_t> w_rowptr_h;          // row pointer of W = A^T A (empty when not built)
  bool stage_values = false;                // single launches stage the CG loop's entry values too
  int kernel_kind = 0;                      // solver kernel variant of single launches (kKernel*)
  int entries_per_lane = 0;                 // A p gather: entries per lane of a row unit
  double kappa_est = 0.0;                   // rank check's kappa(A) estimate (0: not checked)
  double* d_stage_rhs_x = nullptr;          // fct_plan_rhs: scratch iterate of the first stage
  bool dirty_state = false;
  // DCT passes on the tensor cores (grids with a long axis; null when none):
  // host description and device tables shared with clones, own workspace
  std::shared_ptr<TcHost> tc;
  std::shared_ptr<TcDevice> tc_dev;
  std::shared_ptr<TcWork> tc_work;
};

namespace {

fct_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(FCT_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
    return fail(FCT_ERR_NO_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
  return fail(FCT_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FCT_CUDA(call)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Variants of the team solver kernel: plain; kKernelStaged also stages the
// CG loop's entry values in shared memory (single transforms whose tables
// fit); kKernelDeep stages twice as many gather entries per lane and round
// (single transforms of plans with wide rows or many grids, whose tables
// stream from DRAM).  See choose_shape.
enum { kKernelPlain = 0, kKernelStaged = 1, kKernelDeep = 2 };

template <int BT>
const void* kernel_ptr(int kind) {
  if (kind == kKernelStaged) return reinterpret_cast<const void*>(&fct_solve_kernel<BT, true, 0>);
  if (kind == kKernelDeep) return reinterpret_cast<const void*>(&fct_solve_kernel<BT, false, 1>);
  return reinterpret_cast<const void*>(&fct_solve_kernel<BT, false, 0>);
}

const void* solve_kernel_for(int bt, int kind = kKernelPlain) {
  switch (bt) {
    case 128: return kernel_ptr<128>(kind);
    case 512: return kernel_ptr<512>(kind);
    default: return kernel_ptr<256>(kind);
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

fct_status launch_solve(fct_plan P, const SolveArgs& args, int grid, cudaStream_t st, int kind = kKernelPlain) {
  // Reset the per-launch header (queue head, error flag); team barriers are
  // self-cleaning and re-zeroed only after an abandoned launch.
  // Single-transform launches need no reset (team counters reset themselves at
  // exit); batched launches reset the queue head; after an abandoned launch
  // the whole state is cleared.
  if (P->dirty_state) {
    FCT_CUDA(cudaMemsetAsync(args.ls, 0, sizeof(LaunchState), st));
  } else if (args.jobs != nullptr) {
    FCT_CUDA(cudaMemsetAsync(args.ls, 0, offsetof(LaunchState, team_job), st));
  }
  P->dirty_state = false;
  void* kargs[] = {const_cast<SolveArgs*>(&args)};
  FCT_CUDA(cudaLaunchCooperativeKernel(solve_kernel_for(P->block_threads, kind), dim3(grid),
                                       dim3(P->block_threads), kargs,
                                       static_cast<size_t>(args.smem_bytes), st));
  return FCT_OK;
}

// Shared memory (bytes) a block of rank `rank` in a team of G blocks needs to
// stage its table share (see load_block_tabs).
size_t block_smem_need(const fct_plan P, int G, int rank, bool with_values) {
  const DevPlan& hp = P->hp;
  size_t ints = 0;
  int nA = 0, nB = 0;
  // staged entry values: FP32 for the mixed path's inner loop, FP64 otherwise,
  // each after its unit's indices at an 8-byte boundary (one int of padding)
  const size_t wi = with_values ? (P->opt.precision == FCT_MIXED ? 1 : 2) : 0;
  for (int u = rank; u < hp.n_row_units; u += G, ++nA) {
    const int r0 = P->ru_first[u], r1 = P->ru_first[u + 1];
    const size_t ne = static_cast<size_t>(P->rowptr_h[r1] - P->rowptr_h[r0]);
    ints += (r1 - r0 + 1) + ne + 1 + wi * ne;
  }
  for (int c = rank; c < hp.n_coef_chunks; c += G, ++nB)
    ints += static_cast<size_t>(hp.K) * hp.coefs_per_chunk * (1 + wi) + 1;
  int nW = 0;
  if (hp.n_w_units > 0 && P->opt.precision == FCT_MIXED)
    for (int u = rank; u < hp.n_w_units; u += G, ++nW) {
      const int r0 = u * hp.w_rows_per_unit, r1 = std::min(hp.N, r0 + hp.w_rows_per_unit);
      ints += (r1 - r0 + 1) + 2 * static_cast<size_t>(P->w_rowptr_h[r1] - P->w_rowptr_h[r0]);
    }
  ints += 5 * nA + nB + 2 * nW + 1;
  const size_t cmb = hp.coef_split ? coef_combine_bytes(P->block_threads) : 0;
  return cmb + static_cast<size_t>(hp.mats_smem) * sizeof(double) + 4 * ints;
}

size_t team_smem_need(const fct_plan P, int G, bool with_values) {
  size_t need = 0;
  for (int r = 0; r < G; ++r) need = std::max(need, block_smem_need(P, G, r, with_values));
  return need;
}

// Dynamic shared memory of a launch with teams of G blocks that stages only
// the index tables (batches, serving, the condition probe).
size_t launch_smem(const fct_plan P, int G, size_t cap) { return std::min(team_smem_need(P, G, false), cap); }

// Dynamic shared memory a solver block may take without lowering the blocks
// per SM of the plain kernel (the largest static shared memory of the
// kernel variants counted), set as every variant's limit.  Plans and servers
// of one block size compute the same value, so neither lowers the other's
// launch limit.
fct_status solver_smem_cap(int bt, const cudaDeviceProp& prop, int* cap_out, int* per_sm_out) {
  const void* kfn = solve_kernel_for(bt);
  cudaFuncAttributes fa;
  FCT_CUDA(cudaFuncGetAttributes(&fa, kfn));
  for (int kind : {kKernelStaged, kKernelDeep}) {
    cudaFuncAttributes fk;
    FCT_CUDA(cudaFuncGetAttributes(&fk, solve_kernel_for(bt, kind)));
    fa.sharedSizeBytes = std::max(fa.sharedSizeBytes, fk.sharedSizeBytes);
  }
  int per_sm = 0;
  FCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, bt, 0));
  if (per_sm < 1) return fail(FCT_ERR_CUDA, "solver kernel cannot be resident");
  const int reserve = 1024;  // per-block system reservation
  int cap = static_cast<int>(prop.sharedMemPerMultiprocessor / per_sm) - reserve - static_cast<int>(fa.sharedSizeBytes);
  cap = std::min(cap, static_cast<int>(prop.sharedMemPerBlockOptin) - static_cast<int>(fa.sharedSizeBytes));
  cap = std::max(cap, 0) & ~15;
  for (int kind : {kKernelPlain, kKernelStaged, kKernelDeep})
    FCT_CUDA(cudaFuncSetAttribute(solve_kernel_for(bt, kind), cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  *cap_out = cap;
  *per_sm_out = per_sm;
  return FCT_OK;
}

fct_status choose_shape(fct_plan P) {
  int dev = 0;
  FCT_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  FCT_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!prop.cooperativeLaunch) return fail(FCT_ERR_CUDA, "device does not support cooperative launch");
  const void* kfn = solve_kernel_for(P->block_threads);
  int cap = 0, per_sm = 0;
  const fct_status cs = solver_smem_cap(P->block_threads, prop, &cap, &per_sm);
  if (cs != FCT_OK) return cs;
  if (P->hp.coef_split && cap < coef_combine_bytes(P->block_threads))
    return fail(FCT_ERR_CUDA, "no shared memory for the grid-split gather");
  P->blocks_per_sm = per_sm;
  P->smem_cap = cap;
  P->max_coresident = per_sm * prop.multiProcessorCount;
  int units = std::max({P->hp.n_row_units, P->hp.n_coef_chunks, P->hp.n_rowel_chunks, 1});
  for (int p = 0; p < P->H.npass; ++p)
    units = std::max(units, P->H.pass_chunk_off[p + 1] - P->H.pass_chunk_off[p]);
  int g = std::min(P->max_coresident, units);
  if (P->opt.max_blocks > 0) g = std::min(g, P->opt.max_blocks);
  P->grid_blocks = std::max(g, 1);
  // A single transform on the whole GPU also stages the entry values of the
  // CG loop when every block's share fits (fct_solve_kernel<BT, true>).
  const size_t need_values = team_smem_need(P, P->grid_blocks, true);
  P->stage_values = need_values <= static_cast<size_t>(cap);
  P->smem_bytes = static_cast<int>((P->stage_values ? need_values : launch_smem(P, P->grid_blocks, cap)) + 15) & ~15;
  P->smem_bytes = std::min(P->smem_bytes, cap);
  int chk = 0;
  FCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&chk, kfn, P->block_threads, P->smem_bytes));
  if (chk * prop.multiProcessorCount < P->grid_blocks) return fail(FCT_ERR_CUDA, "solver grid does not fit");
  if (P->stage_values) {
    FCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&chk, solve_kernel_for(P->block_threads, kKernelStaged),
                                                           P->block_threads, P->smem_bytes));
    if (chk * prop.multiProcessorCount < P->grid_blocks) P->stage_values = false;
  }
  P->kernel_kind = P->stage_values ? kKernelStaged : kKernelPlain;
  if (!P->stage_values && (P->hp.n_wide_units > 0 || P->K >= 64)) {
    FCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&chk, solve_kernel_for(P->block_threads, kKernelDeep),
                                                           P->block_threads, P->smem_bytes));
    if (chk * prop.multiProcessorCount >= P->grid_blocks) P->kernel_kind = kKernelDeep;
  }
  return FCT_OK;
}

SolveJob make_job(fct_plan P, const double* samples, double* coeffs, fct_report* drep) {
  SolveJob j{};
  j.plan = P->dp;
  j.samples = samples;
  j.coeffs = coeffs;
  j.report = drep;
  j.precision = P->opt.precision;
  j.max_iter = P->opt.max_iter;
  j.max_refine = P->opt.max_refine;
  j.tol = P->opt.tol;
  j.inner_tol = P->opt.inner_tol;
  return j;
}

unsigned long long timeout_ns(fct_plan P);

// Single-transform executes of plans with tensor-core grids: their DCT passes
// run first (same stream), and the job skips them (kJobTcDct).
fct_status run_tc_passes(fct_plan P, const double* samples, cudaStream_t st, SolveJob* job) {
  if (!P->tc) return FCT_OK;
  const fct_status s = tc_run(*P->tc, *P->tc_dev, *P->tc_work, samples, P->hp.y0, P->hp.y1, &P->ls->err,
                              timeout_ns(P), st);
  if (s != FCT_OK) return s;
  job->flags |= kJobTcDct;
  return FCT_OK;
}

unsigned long long timeout_ns(fct_plan P) {
  double t = P->opt.timeout_s > 0 ? P->opt.timeout_s : 4.0;
  return static_cast<unsigned long long>(t * 1e9);
}

}  // namespace

extern "C" {

// Condition estimate of a finished plan for its rank check: kRankCheckIterations
// Lanczos steps of fct_plan_condition from a fixed pseudo-random start
// (splitmix64 of the index, uniform in [-1, 1)); scratch is taken and
// returned on the plan's build stream.
constexpr int kRankCheckIterations = 200;
static fct_status rank_check(fct_plan P, cudaStream_t cs, double* kappa, double* lmin) {
  const int64_t N = P->N;
  std::vector<double> h(static_cast<size_t>(N));
  for (int64_t i = 0; i < N; ++i) {
    uint64_t z = static_cast<uint64_t>(i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    h[static_cast<size_t>(i)] = static_cast<double>(z >> 11) * 0x1.0p-52 - 1.0;
  }
  double* d = nullptr;
  FCT_CUDA(cudaMallocAsync(&d, sizeof(double) * 2 * N, cs));
  cudaError_t e = cudaMemcpyAsync(d, h.data(), sizeof(double) * N, cudaMemcpyHostToDevice, cs);
  fct_status s = e == cudaSuccess ? FCT_OK : cuda_fail(e, "rank check upload");
  int used = 0;
  if (s == FCT_OK) s = fct_plan_condition(P, d, d + N, kRankCheckIterations, kappa, lmin, nullptr, &used, cs);
  cudaFreeAsync(d, cs);
  e = cudaStreamSynchronize(cs);
  if (s == FCT_OK && e != cudaSuccess) s = cuda_fail(e, "rank check");
  return s;
}

fct_status fct_plan_create(fct_plan* out, int D, int64_t N, const uint16_t* support, int K, const int32_t* sizes,
                           const double* nodes, const fct_options* opt) {
  if (!out) return fail(FCT_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  fct_options o;
  fct_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != FCT_FP64 && o.precision != FCT_MIXED) return fail(FCT_ERR_INVALID_ARG, "bad precision");
  if (!(o.tol > 0.0) || o.max_iter < 1 || o.max_refine < 0 || !(o.inner_tol > 0.0))
    return fail(FCT_ERR_INVALID_ARG, "bad tolerance or iteration cap");
  if (o.block_threads == 0) o.block_threads = 256;
  if (o.block_threads != 128 && o.block_threads != 256 && o.block_threads != 512)
    return fail(FCT_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
  if (o.coef_lanes != 0 && (o.coef_lanes < 1 || o.coef_lanes > 16 || (o.coef_lanes & (o.coef_lanes - 1))))
    return fail(FCT_ERR_INVALID_ARG, "coef_lanes must be 0 or a power of two <= 16");
  if (o.coef_split < -1 || o.coef_split > 1) return fail(FCT_ERR_INVALID_ARG, "coef_split must be -1, 0 or 1");
  if (!(o.kappa_max >= 0.0)) return fail(FCT_ERR_INVALID_ARG, "kappa_max must be >= 0 (0 = no rank check)");
  if (o.entries_per_lane != 0 && o.entries_per_lane != 2 && o.entries_per_lane != 4 && o.entries_per_lane != 8)
    return fail(FCT_ERR_INVALID_ARG, "entries_per_lane must be 0, 2, 4 or 8");
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1) return fail(FCT_ERR_NO_DEVICE, "no CUDA device");

  if (o.plan_build < 0 || o.plan_build > 2) return fail(FCT_ERR_INVALID_ARG, "plan_build must be 0, 1 or 2");
  const bool on_device = o.plan_build != FCT_PLAN_BUILD_HOST;

  // Plan construction runs on a stream of its own and synchronises only that
  // stream, so plans can be built while other streams keep the device busy
  // (e.g. a serving launch, when it leaves SMs free).
  cudaStream_t cs = nullptr;
  ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return cuda_fail(ce, "plan stream");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } stream_guard{cs};
  auto* P = new fct_plan_s();
  P->opt = o;
  std::string err;
  fct_status s = build_host_tables(D, N, support, K, sizes, nodes, o.grid_kind, true, &P->H, &err, !on_device);
  if (s != FCT_OK) {
    delete P;
    return fail(s, err);
  }
  HostTables& H = P->H;
  P->D = D;
  P->K = K;
  P->N = N;
  P->M = H.M;
  P->sizes.assign(sizes, sizes + static_cast<size_t>(K) * D);
  for (int64_t e = 0; e < N * D; ++e) P->dmax = std::max<int>(P->dmax, support[e]);
  P->block_threads = o.block_threads;
  cudaGetDevice(&P->device);

  // launch shape of the solver: warp 0 of each block reduces, the other
  // BT - 32 threads gather
  const int BT = o.block_threads;
  const int workers = BT - 32;
  int L = o.coef_lanes;
  if (L == 0) {
    // at most 8 grid entries per lane, so one staged round of loads
    L = 1;
    while (L < 16 && L * 8 < K) L <<= 1;
  }
  // Entries per gather lane: the smallest of 2, 4, 8 whose row units fit in
  // one wave of co-resident blocks (a block with two units while others have
  // one makes everybody wait at the next barrier).
  int epl = 8;
  int64_t wave = 0;  // co-resident blocks of the solver kernel
  {
    int per_sm = 0, nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_kernel_for(BT), BT, 0) == cudaSuccess)
      wave = static_cast<int64_t>(per_sm) * nsm;
  }
  DeviceTables DT;  // device-built tables (scratch, freed on return)
  if (on_device) {
    s = build_device_tables(&H, support, sizes, nodes, o.grid_kind, workers, wave, o.entries_per_lane, &epl, &DT,
                            cs);
    if (s != FCT_OK) {
      delete P;
      return s;
    }
  } else {
    int64_t classes[3][kLaneClasses];
    lane_class_counts(H, classes);
    epl = pick_entries_per_lane(classes, workers, wave, o.entries_per_lane);
    device_row_order(&H, epl);
  }
  // tensor-core DCT passes: which grids, their A slices and pass lists (may
  // add the identity matrix to the DCT matrices, so before their upload)
  if (o.tensor_dct < -1 || o.tensor_dct > 1) {
    delete P;
    return fail(FCT_ERR_INVALID_ARG, "tensor_dct must be -1, 0 or 1");
  }
  {
    auto T = std::make_shared<TcHost>();
    s = build_tc_host(&H, sizes, o.grid_kind, o.tensor_dct, T.get());
    if (s != FCT_OK) {
      delete P;
      return fail(s, "tensor-core DCT set-up: a pass is too large");
    }
    if (!T->empty()) P->tc = T;
  }
  P->R = H.R;
  DevPlan& hp = P->hp;
  hp.N = static_cast<int32_t>(N);
  hp.R = static_cast<int32_t>(H.R);
  hp.K = K;
  hp.D = D;
  hp.M = H.M;
  hp.npass = H.npass;
  // grid-split A^T q gather: coalesced reads of the coefficient-major tables
  // (32 consecutive coefficients per warp load), and a warp's q reads fall in
  // one grid's rows; pays where each coefficient has many grids
  const bool split = o.coef_split > 0 || (o.coef_split == 0 && K >= kCoefSplitMinGrids);
  hp.coef_split = split ? 1 : 0;
  hp.coef_lanes = split ? 1 : L;
  hp.workers = workers;
  hp.coefs_per_chunk = split ? 32 : workers / L;
  hp.n_coef_chunks = static_cast<int32_t>((N + hp.coefs_per_chunk - 1) / hp.coefs_per_chunk);
  hp.n_rowel_chunks = static_cast<int32_t>((H.R + BT - 1) / BT);
  std::vector<int32_t> ru_first, ru_lanes, rowbase, rowk;
  row_units(H, workers, epl, &ru_first, &ru_lanes);
  P->entries_per_lane = epl;
  if (!on_device) final_pass_rows(H, &rowbase, &rowk);  // the device build made them
  hp.n_row_units = static_cast<int32_t>(ru_lanes.size());
  hp.n_wide_units = 0;
  while (hp.n_wide_units < hp.n_row_units && ru_lanes[hp.n_wide_units] > 32) ++hp.n_wide_units;
  for (int32_t u = hp.n_wide_units; u < hp.n_row_units; ++u)
    if (ru_lanes[u] > 32) {
      delete P;
      return fail(FCT_ERR_INVALID_ARG, "internal: wide row units must come first");
    }
  hp.n_mats = static_cast<int32_t>(H.dct_mats.size());
  hp.mats_smem = H.dct_mats.size() * sizeof(double) <= 32768 ? hp.n_mats : 0;
  P->ru_first = ru_first;
  P->rowptr_h = H.rowptr;

  // Normal matrix W = A^T A for the mixed path's inner solve (one team barrier
  // per iteration instead of two).  Auto: only where W is small next to A.
  std::vector<int32_t> w_rowptr, w_col;
  std::vector<float> w_val32;
  {
    const int64_t KN2 = 2 * static_cast<int64_t>(K) * N;
    const int64_t bound = normal_matrix_bound(H);
    bool want = o.normal_matrix > 0 ||
                (o.normal_matrix == 0 && o.precision == FCT_MIXED && bound <= 2 * KN2);
    if (o.normal_matrix > 0 && bound > (int64_t{1} << 30)) {
      delete P;
      return fail(FCT_ERR_INVALID_ARG, "normal_matrix = 1 but A^T A would exceed 2^30 nonzeros");
    }
    if (want && N > 0 && on_device) {
      s = download_device_tables(DT, &H);
      if (s != FCT_OK) {
        delete P;
        return s;
      }
    }
    if (want && N > 0) {
      std::vector<double> wv64;
      normal_matrix(H, &w_rowptr, &w_col, &wv64);
      const int64_t nnz = static_cast<int64_t>(w_col.size());
      if (o.normal_matrix == 0 && (nnz > KN2 || nnz > 8000000)) {
        w_rowptr.clear();
        w_col.clear();
      } else {
        w_val32.resize(nnz);
        for (int64_t i = 0; i < nnz; ++i) w_val32[i] = static_cast<float>(wv64[i]);
      }
    }
    if (!w_col.empty()) {
      // lanes per row: as many as keep the units within one wave, at most half
      // the mean row length
      int LW = 32;
      const int64_t wv = wave > 0 ? wave : 1;
      while (LW > 1 && (N + workers / LW - 1) / (workers / LW) > wv) LW >>= 1;
      const double mean_row = static_cast<double>(w_col.size()) / static_cast<double>(N);
      while (LW > 1 && 2.0 * LW > mean_row) LW >>= 1;
      hp.w_lanes = LW;
      hp.w_rows_per_unit = workers / LW;
      hp.n_w_units = static_cast<int32_t>((N + hp.w_rows_per_unit - 1) / hp.w_rows_per_unit);
    }
  }
  const int64_t nnzw = static_cast<int64_t>(w_col.size());
  P->w_rowptr_h = w_rowptr;

  // one device allocation, carved in 256-byte aligned pieces
  const int64_t KN = static_cast<int64_t>(K) * N;
  const int64_t nnodes = static_cast<int64_t>(H.node_pos.size());
  struct Piece {
    void** dst;
    size_t bytes;
  };
  std::vector<Piece> pieces;
  auto add = [&](void* dst, size_t bytes) { pieces.push_back({reinterpret_cast<void**>(dst), bytes}); };
  int32_t *d_pass, *d_rowptr, *d_col, *d_crow, *d_rowbase, *d_rowk, *d_rowgrid, *d_ru_first, *d_ru_lanes;
  DctChunk* d_chunks;
  GridFinal* d_gfinal;
  double *d_mats, *d_wcsr, *d_wcm;
  float *d_wcsr32, *d_wcm32;
  add(&P->dp, sizeof(DevPlan));
  add(&P->ls, sizeof(LaunchState));
  add(&P->drep, sizeof(fct_report));
  add(&d_pass, sizeof(int32_t) * H.pass_chunk_off.size());
  add(&d_chunks, sizeof(DctChunk) * H.dct_chunks.size());
  add(&d_mats, sizeof(double) * H.dct_mats.size());
  add(&d_gfinal, sizeof(GridFinal) * K);
  add(&d_rowbase, sizeof(int32_t) * H.R);
  add(&d_rowk, sizeof(int32_t) * H.R);
  add(&d_rowgrid, sizeof(int32_t) * H.R);
  add(&d_ru_first, sizeof(int32_t) * ru_first.size());
  add(&d_ru_lanes, sizeof(int32_t) * ru_lanes.size());
  add(&d_rowptr, sizeof(int32_t) * (H.R + 1));
  add(&d_col, sizeof(int32_t) * KN);
  add(&d_wcsr, sizeof(double) * KN);
  add(&d_wcsr32, sizeof(float) * KN);
  add(&d_crow, sizeof(int32_t) * KN);
  add(&d_wcm, sizeof(double) * KN);
  add(&d_wcm32, sizeof(float) * KN);
  int32_t *d_wrowptr, *d_wcol;
  float* d_wval;
  add(&d_wrowptr, sizeof(int32_t) * (nnzw > 0 ? N + 1 : 1));
  add(&d_wcol, sizeof(int32_t) * nnzw);
  add(&d_wval, sizeof(float) * nnzw);
  add(&hp.y0, sizeof(double) * std::max<int64_t>(H.M, 1));
  add(&hp.y1, sizeof(double) * std::max<int64_t>(H.M, 1));
  add(&hp.b, sizeof(double) * H.R);
  add(&hp.rres, sizeof(double) * H.R);
  add(&hp.q, sizeof(double) * H.R);
  add(&hp.sp, sizeof(double2) * N);
  add(&hp.part_r, sizeof(double) * hp.n_row_units);
  add(&hp.part_c, sizeof(double) * hp.n_coef_chunks);
  add(&hp.q32, sizeof(float) * H.R);
  add(&hp.sp32, sizeof(float2) * N);
  add(&hp.dx32, sizeof(float) * N);
  add(&hp.wv, sizeof(float) * (hp.n_w_units > 0 ? 6 * N : 1));
  add(&hp.pw64, sizeof(double2) * 2 * std::max(hp.n_w_units, 1));
  add(&P->d_sizes, sizeof(int32_t) * K * D);
  add(&P->d_offsets, sizeof(int64_t) * (K + 1));
  add(&P->d_node_off, sizeof(int32_t) * K * D);
  add(&P->d_node_pos, sizeof(double) * nnodes);
  add(&P->d_support, sizeof(uint16_t) * N * D);
  add(&P->d_ttab, sizeof(double) * nnodes * (P->dmax + 1));
  add(&P->d_ichunks, sizeof(DctChunk) * H.idct_chunks.size());
  add(&P->d_emats, sizeof(double) * H.eval_mats.size());
  size_t total = 0;
  for (auto& pc : pieces) total += align256(std::max<size_t>(pc.bytes, 1));
  cudaError_t e = cudaMalloc(&P->dmem, total);
  if (e != cudaSuccess) {
    delete P;
    return cuda_fail(e, "cudaMalloc(plan)");
  }
  P->dbytes = total;
  P->tables = std::shared_ptr<char>(P->dmem, [](char* p) { cudaFree(p); });
  {
    size_t off = 0;
    for (auto& pc : pieces) {
      *pc.dst = P->dmem + off;
      off += align256(std::max<size_t>(pc.bytes, 1));
    }
  }
  hp.pass_chunk_off = d_pass;
  hp.dct_chunks = d_chunks;
  hp.dct_mats = d_mats;
  hp.gfinal = d_gfinal;
  hp.rowbase = d_rowbase;
  hp.rowk = d_rowk;
  hp.rowgrid = d_rowgrid;
  hp.ru_first = d_ru_first;
  hp.ru_lanes = d_ru_lanes;
  hp.rowptr = d_rowptr;
  hp.col = d_col;
  hp.wcsr = d_wcsr;
  hp.wcsr32 = d_wcsr32;
  hp.crow = d_crow;
  hp.wcm = d_wcm;
  hp.wcm32 = d_wcm32;
  hp.wrowptr = d_wrowptr;
  hp.wcol = d_wcol;
  hp.wval = d_wval;

  std::vector<float> w32, wc32;
  if (!on_device) {
    w32.resize(KN);
    wc32.resize(KN);
    for (int64_t i = 0; i < KN; ++i) {
      w32[i] = static_cast<float>(H.wcsr[i]);
      wc32[i] = static_cast<float>(H.weight[i]);
    }
  }
  auto up = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDefault : cudaMemcpyHostToDevice, cs);
  };
  cudaError_t ue = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (ue == cudaSuccess) ue = x;
  };
  chk(cudaMemsetAsync(P->ls, 0, sizeof(LaunchState), cs));
  chk(up(d_pass, H.pass_chunk_off.data(), sizeof(int32_t) * H.pass_chunk_off.size()));
  chk(up(d_chunks, H.dct_chunks.data(), sizeof(DctChunk) * H.dct_chunks.size()));
  chk(up(d_mats, H.dct_mats.data(), sizeof(double) * H.dct_mats.size()));
  chk(up(d_gfinal, H.gfinal.data(), sizeof(GridFinal) * K));
  chk(up(d_rowbase, on_device ? static_cast<const void*>(DT.rowbase) : rowbase.data(), sizeof(int32_t) * H.R));
  chk(up(d_rowk, on_device ? static_cast<const void*>(DT.rowk) : rowk.data(), sizeof(int32_t) * H.R));
  chk(up(d_rowgrid, on_device ? static_cast<const void*>(DT.rowgrid) : H.rowgrid.data(), sizeof(int32_t) * H.R));
  chk(up(d_ru_first, ru_first.data(), sizeof(int32_t) * ru_first.size()));
  chk(up(d_ru_lanes, ru_lanes.data(), sizeof(int32_t) * ru_lanes.size()));
  chk(up(d_rowptr, H.rowptr.data(), sizeof(int32_t) * (H.R + 1)));
  // alias tables (the coefficient-major row table holds global rows): from
  // the device build's scratch, or from the host tables
  chk(up(d_col, on_device ? static_cast<const void*>(DT.col) : H.col.data(), sizeof(int32_t) * KN));
  chk(up(d_wcsr, on_device ? static_cast<const void*>(DT.wcsr) : H.wcsr.data(), sizeof(double) * KN));
  chk(up(d_wcsr32, on_device ? static_cast<const void*>(DT.wcsr32) : w32.data(), sizeof(float) * KN));
  chk(up(d_crow, on_device ? static_cast<const void*>(DT.crow) : H.crow.data(), sizeof(int32_t) * KN));
  chk(up(d_wcm, on_device ? static_cast<const void*>(DT.wcm) : H.weight.data(), sizeof(double) * KN));
  chk(up(d_wcm32, on_device ? static_cast<const void*>(DT.wcm32) : wc32.data(), sizeof(float) * KN));
  DT.release();
  if (nnzw > 0) {
    chk(up(d_wrowptr, w_rowptr.data(), sizeof(int32_t) * (N + 1)));
    chk(up(d_wcol, w_col.data(), sizeof(int32_t) * nnzw));
    chk(up(d_wval, w_val32.data(), sizeof(float) * nnzw));
  }
  chk(up(P->d_sizes, sizes, sizeof(int32_t) * K * D));
  chk(up(P->d_offsets, H.offsets.data(), sizeof(int64_t) * (K + 1)));
  chk(up(P->d_node_off, H.node_off.data(), sizeof(int32_t) * K * D));
  chk(up(P->d_node_pos, H.node_pos.data(), sizeof(double) * nnodes));
  chk(up(P->d_support, support, sizeof(uint16_t) * N * D));
  chk(up(P->d_ichunks, H.idct_chunks.data(), sizeof(DctChunk) * H.idct_chunks.size()));
  chk(up(P->d_emats, H.eval_mats.data(), sizeof(double) * H.eval_mats.size()));
  s = FCT_OK;
  if (ue == cudaSuccess && P->tc) {
    std::vector<int32_t> rb, rk;
    final_pass_rows_for(H, P->tc->gfinal, &rb, &rk);
    auto dev = std::make_shared<TcDevice>();
    auto wk = std::make_shared<TcWork>();
    s = tc_upload(*P->tc, rb, rk, dev.get());
    if (s == FCT_OK) s = tc_alloc_work(*P->tc, wk.get());
    if (s == FCT_OK) {
      P->tc_dev = dev;
      P->tc_work = wk;
      hp.npass_tc = P->tc->npass_fp64;
      hp.pass_chunk_off_tc = dev->pass_chunk_off;
      hp.dct_chunks_tc = dev->dct_chunks;
      hp.gfinal_tc = dev->gfinal;
      hp.rowbase_tc = dev->rowbase;
      hp.rowk_tc = dev->rowk;
      P->tc->a_bits.clear();
      P->tc->a_bits.shrink_to_fit();
    }
  }
  if (ue == cudaSuccess && s == FCT_OK) s = choose_shape(P);
  if (ue == cudaSuccess && s == FCT_OK) chk(up(P->dp, &hp, sizeof(DevPlan)));
  if (ue == cudaSuccess && s == FCT_OK && nnodes > 0) {
    cheb_table_kernel<<<static_cast<unsigned>((nnodes + 127) / 128), 128, 0, cs>>>(
        P->d_node_pos, static_cast<int>(nnodes), P->dmax, P->d_ttab);
    chk(cudaGetLastError());
  }
  chk(cudaStreamSynchronize(cs));
  if (ue != cudaSuccess || s != FCT_OK) {
    P->tables.reset();
    delete P;
    return ue != cudaSuccess ? cuda_fail(ue, "plan upload") : s;
  }
  // free the host copies that are no longer needed
  H.bin.clear(); H.bin.shrink_to_fit();
  H.col.clear(); H.col.shrink_to_fit();
  H.wcsr.clear(); H.wcsr.shrink_to_fit();
  H.weight.clear(); H.weight.shrink_to_fit();
  H.crow.clear(); H.crow.shrink_to_fit();
  if (o.kappa_max > 0.0) {
    // Algorithm 2's acceptance test on the finished plan: refuse it when the
    // Lanczos estimate of kappa(A) exceeds the bound (a rank-deficient A has
    // a zero Ritz value, so its estimate is unbounded)
    double kappa = 0.0, lmin = 0.0;
    s = rank_check(P, cs, &kappa, &lmin);
    if (s != FCT_OK) {
      fct_destroy(P);
      return s;
    }
    if (!(lmin > 0.0) || !(kappa <= o.kappa_max)) {
      fct_destroy(P);
      return fail(FCT_ERR_RANK, "kappa(A) estimate " + std::to_string(kappa) + " exceeds kappa_max " +
                                    std::to_string(o.kappa_max) + " (or A is rank-deficient)");
    }
    P->kappa_est = kappa;
  }
  *out = P;
  return FCT_OK;
}

fct_status fct_plan_tables(fct_plan P, int32_t* rowptr, int32_t* col, double* wcsr, int32_t* crow, double* wcm,
                           int64_t* bins) {
  if (!P) return fail(FCT_ERR_INVALID_ARG, "NULL plan");
  const int64_t KN = static_cast<int64_t>(P->K) * P->N, R = P->R;
  cudaError_t ue = cudaSuccess;
  auto down = [&](void* dst, const void* src, size_t bytes) {
    if (dst && ue == cudaSuccess) ue = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
  };
  down(rowptr, P->hp.rowptr, sizeof(int32_t) * (R + 1));
  down(col, P->hp.col, sizeof(int32_t) * KN);
  down(wcsr, P->hp.wcsr, sizeof(double) * KN);
  down(crow, P->hp.crow, sizeof(int32_t) * KN);
  down(wcm, P->hp.wcm, sizeof(double) * KN);
  if (ue != cudaSuccess) return cuda_fail(ue, "fct_plan_tables");
  if (bins)
    for (int64_t r = 0; r < R; ++r) bins[r] = P->H.rowsrc[r];
  return FCT_OK;
}

fct_status fct_plan_get_info(fct_plan P, fct_plan_info* info) {
  if (!P || !info) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  info->N = P->N;
  info->M = P->M;
  info->R = P->R;
  info->nnz = static_cast<int64_t>(P->K) * P->N;
  info->D = P->D;
  info->K = P->K;
  info->passes = P->H.npass;
  info->grid_blocks = P->grid_blocks;
  info->block_threads = P->block_threads;
  info->coef_lanes = P->hp.coef_lanes;
  info->device_bytes = static_cast<int64_t>(P->dbytes);
  info->normal_nnz = P->hp.n_w_units > 0 ? static_cast<int64_t>(P->w_rowptr_h.back()) : 0;
  info->coef_split = P->hp.coef_split;
  info->row_units = P->hp.n_row_units;
  info->wide_rows = P->hp.n_wide_units;
  info->coef_chunks = P->hp.n_coef_chunks;
  info->entries_per_lane = P->entries_per_lane;
  info->kappa_estimate = P->kappa_est;
  info->kernel_variant = P->kernel_kind;
  info->tensor_dct_grids = 0;
  info->tensor_dct_flops = 0;
  if (P->tc) {
    for (char g : P->tc->grid_tc) info->tensor_dct_grids += g ? 1 : 0;
    // every GEMM tile issues 36 digit-slice products (M 128, N 64, K 16) per K step
    const int64_t per_step = 36ll * 2 * kTcM * kTcN * kTcK;
    for (size_t t = 0; t + 3 < P->tc->gemm_tasks.size(); t += 4)
      info->tensor_dct_flops += per_step * P->tc->gp[P->tc->gemm_tasks[t]].ksteps;
  }
  return FCT_OK;
}

fct_status fct_grid_offsets(fct_plan P, int64_t* offsets) {
  if (!P || !offsets) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(offsets, P->H.offsets.data(), sizeof(int64_t) * (P->K + 1));
  return FCT_OK;
}

fct_status fct_evaluate(fct_plan P, const double* coeffs, int64_t npoints, const double* points, double* values,
                        void* stream) {
  if (!P || npoints < 0) return fail(FCT_ERR_INVALID_ARG, "NULL plan or negative point count");
  if (npoints == 0) return FCT_OK;
  if (!coeffs || !points || !values) return fail(FCT_ERR_INVALID_ARG, "NULL buffer");
  const size_t per_point = sizeof(double) * static_cast<size_t>(P->D) * (P->dmax + 1);
  const size_t fixed = sizeof(double) * kEvalTile + sizeof(uint16_t) * kEvalTile * static_cast<size_t>(P->D);
  int dev = 0, optin = 0;
  FCT_CUDA(cudaGetDevice(&dev));
  FCT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  int ppb = 8;
  while (ppb > 1 && fixed + ppb * per_point > static_cast<size_t>(optin)) ppb >>= 1;
  const size_t smem = fixed + ppb * per_point;
  if (smem > static_cast<size_t>(optin))
    return fail(FCT_ERR_INVALID_ARG, "D x (max degree + 1) too large for the evaluation tables");
  FCT_CUDA(cudaFuncSetAttribute(eval_expansion_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem)));
  const int64_t blocks = (npoints + ppb - 1) / ppb;
  if (blocks > 0x7fffffff) return fail(FCT_ERR_INVALID_ARG, "too many points");
  eval_expansion_kernel<<<static_cast<unsigned>(blocks), 32 * ppb, smem, static_cast<cudaStream_t>(stream)>>>(
      P->d_support, coeffs, static_cast<int>(P->N), P->D, P->dmax, points, npoints, values);
  FCT_CUDA(cudaGetLastError());
  return FCT_OK;
}

fct_status fct_sample(fct_plan P, int family, const double* params, int64_t nparams, double* samples,
                      void* stream) {
  if (!P || !params || !samples) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  const bool force_folded = (family & FCT_SAMPLE_FOLDED) != 0;
  family &= ~FCT_SAMPLE_FOLDED;
  int64_t need = 0;
  switch (family) {
    case FCT_FAMILY_POLY: need = P->N; break;
    case FCT_FAMILY_GAUSSCOS: need = 2 * P->D; break;
    case FCT_FAMILY_RATIONAL: need = P->D; break;
    case FCT_FAMILY_POLY_GAUSSCOS: need = 2 * P->D + P->N; break;
    default: return fail(FCT_ERR_INVALID_ARG, "unknown family");
  }
  if (nparams != need) return fail(FCT_ERR_INVALID_ARG, "params length does not match the family");
  const bool poly = family == FCT_FAMILY_POLY || family == FCT_FAMILY_POLY_GAUSSCOS;
  if (force_folded && !poly) return fail(FCT_ERR_INVALID_ARG, "FCT_SAMPLE_FOLDED applies to polynomial families");
  // term-by-term evaluation costs M*N*D; above this the folded path is used
  const bool folded = poly && (force_folded || static_cast<double>(P->M) * static_cast<double>(P->N) > 4e10);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nparams > P->params_cap) {
    if (P->d_params) {
      FCT_CUDA(cudaStreamSynchronize(st));
      cudaFree(P->d_params);
      P->d_params = nullptr;
    }
    FCT_CUDA(cudaMalloc(&P->d_params, sizeof(double) * nparams));
    P->params_cap = nparams;
  }
  FCT_CUDA(cudaMemcpyAsync(P->d_params, params, sizeof(double) * nparams, cudaMemcpyHostToDevice, st));
  FCT_CUDA(cudaStreamSynchronize(st));  // params are host memory the caller may reuse
  SampleArgs a;
  a.sizes = P->d_sizes;
  a.offsets = P->d_offsets;
  a.node_off = P->d_node_off;
  a.node_pos = P->d_node_pos;
  a.ttab = P->d_ttab;
  a.support = P->d_support;
  a.params = P->d_params;
  a.out = samples;
  a.M = P->M;
  a.K = P->K;
  a.D = P->D;
  a.N = static_cast<int>(P->N);
  a.family = folded ? (family == FCT_FAMILY_POLY_GAUSSCOS ? FCT_FAMILY_GAUSSCOS : -1) : family;
  a.dmax = P->dmax;
  const int bt = 128;
  if (a.family >= 0) {
    sample_kernel<<<static_cast<unsigned>((P->M + bt - 1) / bt), bt, 0, st>>>(a);
    FCT_CUDA(cudaGetLastError());
  }
  if (folded) {
    const double* c = P->d_params + (family == FCT_FAMILY_POLY_GAUSSCOS ? 2 * P->D : 0);
    FCT_CUDA(cudaMemsetAsync(P->hp.y0, 0, sizeof(double) * P->M, st));
    fold_scatter_kernel<<<static_cast<unsigned>((P->R + 255) / 256), 256, 0, st>>>(P->dp, c);
    FCT_CUDA(cudaGetLastError());
    const int add = family == FCT_FAMILY_POLY_GAUSSCOS ? 1 : 0;
    for (int p = 0; p < P->H.nipass; ++p) {
      const int c0 = P->H.ipass_chunk_off[p], c1 = P->H.ipass_chunk_off[p + 1];
      if (c1 > c0) eval_pass_kernel<<<c1 - c0, 256, 0, st>>>(P->dp, P->d_ichunks, c0, P->d_emats, samples, add);
      FCT_CUDA(cudaGetLastError());
    }
  }
  return FCT_OK;
}

static fct_status read_report(fct_plan P, fct_report* dsrc, cudaStream_t st, fct_report* rep, int n = 1) {
  FCT_CUDA(cudaMemcpyAsync(rep, dsrc, sizeof(fct_report) * n, cudaMemcpyDeviceToHost, st));
  FCT_CUDA(cudaStreamSynchronize(st));
  int err = 0;
  FCT_CUDA(cudaMemcpy(&err, &P->ls->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    P->dirty_state = true;
    for (int i = 0; i < n; ++i) rep[i].status = err;
    return fail(static_cast<fct_status>(err), "device-side wait expired in the solver");
  }
  fct_status worst = FCT_OK;
  for (int i = 0; i < n; ++i)
    if (rep[i].status != FCT_OK && worst == FCT_OK) worst = static_cast<fct_status>(rep[i].status);
  if (worst != FCT_OK) return fail(worst, std::string("solver finished with ") + fct_status_string(worst));
  return FCT_OK;
}

fct_status fct_execute(fct_plan P, const double* samples, double* coeffs, void* stream, fct_report* rep) {
  if (!P || !samples || !coeffs) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolveArgs a{};
  a.single = make_job(P, samples, coeffs, P->drep);
  a.jobs = nullptr;
  a.njobs = 1;
  a.team_blocks = P->grid_blocks;
  a.ls = P->ls;
  a.timeout_ns = timeout_ns(P);
  a.smem_bytes = P->smem_bytes;
  fct_status s = run_tc_passes(P, samples, st, &a.single);
  if (s != FCT_OK) return s;
  s = launch_solve(P, a, P->grid_blocks, st, P->kernel_kind);
  if (s != FCT_OK) return s;
  if (rep) return read_report(P, P->drep, st, rep);
  return FCT_OK;
}

fct_status fct_plan_apply(fct_plan P, const double* in, double* out, int transpose, int64_t* bins, void* stream) {
  if (!P || !in || !out) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  const int64_t n = transpose ? P->N : P->R;
  if (n > 0) {
    alias_apply_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        P->dp, in, out, transpose ? 1 : 0);
    FCT_CUDA(cudaGetLastError());
  }
  if (bins)
    for (int64_t r = 0; r < P->R; ++r) bins[r] = P->H.rowsrc[r];
  return FCT_OK;
}

fct_status fct_plan_rhs(fct_plan P, const double* samples, double* b, int64_t* bins, void* stream) {
  if (!P || !samples || !b) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the team kernel's first stage only: DCT passes, b at the nonempty bins, s = A^T b
  SolveArgs a{};
  a.single = make_job(P, samples, P->d_stage_rhs_x ? P->d_stage_rhs_x : nullptr, P->drep);
  if (!P->d_stage_rhs_x) {
    FCT_CUDA(cudaMalloc(&P->d_stage_rhs_x, sizeof(double) * P->N));
    a.single.coeffs = P->d_stage_rhs_x;
  }
  a.single.flags = kJobPrepareOnly;
  a.jobs = nullptr;
  a.njobs = 1;
  a.team_blocks = P->grid_blocks;
  a.ls = P->ls;
  a.timeout_ns = timeout_ns(P);
  a.smem_bytes = P->smem_bytes;
  fct_status s = run_tc_passes(P, samples, st, &a.single);
  if (s != FCT_OK) return s;
  s = launch_solve(P, a, P->grid_blocks, st, P->kernel_kind);
  if (s != FCT_OK) return s;
  FCT_CUDA(cudaMemcpyAsync(b, P->hp.b, sizeof(double) * P->R, cudaMemcpyDeviceToDevice, st));
  FCT_CUDA(cudaStreamSynchronize(st));
  int err = 0;
  FCT_CUDA(cudaMemcpy(&err, &P->ls->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err != 0) {
    P->dirty_state = true;
    return fail(static_cast<fct_status>(err), "fct_plan_rhs: device-side error");
  }
  if (bins)
    for (int64_t r = 0; r < P->R; ++r) bins[r] = P->H.rowsrc[r];
  return FCT_OK;
}

fct_status fct_plan_last_report(fct_plan P, void* stream, fct_report* rep) {
  if (!P || !rep) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  return read_report(P, P->drep, static_cast<cudaStream_t>(stream), rep);
}

fct_status fct_execute_host(fct_plan P, const double* samples_host, double* coeffs_host, void* stream,
                            fct_report* rep) {
  if (!P || !samples_host || !coeffs_host) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!P->d_stage_in) {
    FCT_CUDA(cudaMalloc(&P->d_stage_in, sizeof(double) * P->M));
    FCT_CUDA(cudaMalloc(&P->d_stage_out, sizeof(double) * P->N));
  }
  FCT_CUDA(cudaMemcpyAsync(P->d_stage_in, samples_host, sizeof(double) * P->M, cudaMemcpyHostToDevice, st));
  fct_status s = fct_execute(P, P->d_stage_in, P->d_stage_out, stream, nullptr);
  if (s != FCT_OK) return s;
  FCT_CUDA(cudaMemcpyAsync(coeffs_host, P->d_stage_out, sizeof(double) * P->N, cudaMemcpyDeviceToHost, st));
  if (rep) return read_report(P, P->drep, st, rep);
  FCT_CUDA(cudaStreamSynchronize(st));
  return FCT_OK;
}

// Checks a batch, orders its jobs (largest transforms first: the shortest
// tail for the device work queue) with each job's report at reports + i, and
// fixes the launch shape: blocks per team G, teams, dynamic shared memory.
static fct_status batch_setup(int B, const fct_plan* plans, const double* const* samples, double* const* coeffs,
                              int team_blocks, fct_report* reports, std::vector<SolveJob>* jobs, int* G_out,
                              int* teams_out, int* smem_out) {
  if (B < 1 || !plans || !samples || !coeffs) return fail(FCT_ERR_INVALID_ARG, "bad batch arguments");
  for (int i = 0; i < B; ++i) {
    if (!plans[i] || !samples[i] || !coeffs[i]) return fail(FCT_ERR_INVALID_ARG, "NULL plan or buffer in batch");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(FCT_ERR_INVALID_ARG, "a plan appears twice in one batch");
    if (plans[i]->block_threads != plans[0]->block_threads)
      return fail(FCT_ERR_INVALID_ARG, "all plans of a batch must use the same block_threads");
  }
  fct_plan P0 = plans[0];
  std::vector<int> order(B);
  for (int i = 0; i < B; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return plans[a]->hp.K * static_cast<int64_t>(plans[a]->N) > plans[b]->hp.K * static_cast<int64_t>(plans[b]->N);
  });
  jobs->assign(B, SolveJob{});
  for (int q = 0; q < B; ++q) {
    const int i = order[q];
    (*jobs)[q] = make_job(plans[i], samples[i], coeffs[i], reports + i);
  }
  int G = team_blocks;
  if (G <= 0) {
    int units = 0;
    for (int i = 0; i < B; ++i) units = std::max(units, plans[i]->grid_blocks);
    G = std::max(1, std::min(units, P0->max_coresident / std::max(1, std::min(B, 16))));
  }
  G = std::min(G, P0->max_coresident);
  *teams_out = std::min(std::max(1, P0->max_coresident / G), std::min(B, kMaxTeams));
  *G_out = G;
  size_t need = 0;
  for (int i = 0; i < B; ++i) need = std::max(need, launch_smem(plans[i], G, static_cast<size_t>(P0->smem_cap)));
  *smem_out = std::min(static_cast<int>(std::min<size_t>(need, P0->smem_cap) + 15) & ~15, P0->smem_cap);
  return FCT_OK;
}

fct_status fct_execute_batch(int B, const fct_plan* plans, const double* const* samples, double* const* coeffs,
                             int team_blocks, void* stream, fct_report* reps) {
  if (B < 1 || !plans || !plans[0]) return fail(FCT_ERR_INVALID_ARG, "bad batch arguments");
  fct_plan P0 = plans[0];
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the batch's job array and reports live in plan 0's memory
  if (P0->djobs_cap < B) {
    if (P0->djobs) {
      FCT_CUDA(cudaStreamSynchronize(st));
      cudaFree(P0->djobs);
      P0->djobs = nullptr;
      P0->djobs_cap = 0;
    }
    FCT_CUDA(cudaMalloc(&P0->djobs, (sizeof(SolveJob) + sizeof(fct_report)) * B));
    P0->djobs_cap = B;
  }
  fct_report* dreps = reinterpret_cast<fct_report*>(P0->djobs + P0->djobs_cap);
  std::vector<SolveJob> jobs;
  int G = 0, teams = 0, smem = 0;
  fct_status s = batch_setup(B, plans, samples, coeffs, team_blocks, dreps, &jobs, &G, &teams, &smem);
  if (s != FCT_OK) return s;
  FCT_CUDA(cudaMemcpyAsync(P0->djobs, jobs.data(), sizeof(SolveJob) * B, cudaMemcpyHostToDevice, st));
  FCT_CUDA(cudaStreamSynchronize(st));
  SolveArgs a{};
  a.jobs = P0->djobs;
  a.njobs = B;
  a.team_blocks = G;
  a.ls = P0->ls;
  a.timeout_ns = timeout_ns(P0);
  a.smem_bytes = smem;
  s = launch_solve(P0, a, teams * G, st);
  if (s != FCT_OK) return s;
  if (reps) return read_report(P0, dreps, st, reps, B);
  return FCT_OK;
}

}  // extern "C"

struct fct_batch_s {
  int B = 0, G = 0, teams = 0, smem = 0, block_threads = 0, device = 0;
  unsigned long long tns = 0;
  SolveJob* djobs = nullptr;   // [B] jobs, then [B] reports
  fct_report* dreps = nullptr;
  LaunchState* ls = nullptr;
};

extern "C" {

fct_status fct_batch_create(fct_batch* out, int B, const fct_plan* plans, const double* const* samples,
                            double* const* coeffs, int team_blocks) {
  if (!out) return fail(FCT_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (B < 1 || !plans || !plans[0]) return fail(FCT_ERR_INVALID_ARG, "bad batch arguments");
  auto* Bt = new fct_batch_s();
  auto fail_free = [&](fct_status st) {
    if (Bt->djobs) cudaFree(Bt->djobs);
    if (Bt->ls) cudaFree(Bt->ls);
    delete Bt;
    return st;
  };
  cudaError_t e = cudaMalloc(&Bt->djobs, (sizeof(SolveJob) + sizeof(fct_report)) * B);
  if (e == cudaSuccess) e = cudaMalloc(&Bt->ls, sizeof(LaunchState));
  if (e == cudaSuccess) e = cudaMemset(Bt->ls, 0, sizeof(LaunchState));
  if (e != cudaSuccess) return fail_free(cuda_fail(e, "fct_batch_create"));
  Bt->dreps = reinterpret_cast<fct_report*>(Bt->djobs + B);
  e = cudaMemset(Bt->dreps, 0, sizeof(fct_report) * B);
  if (e != cudaSuccess) return fail_free(cuda_fail(e, "fct_batch_create"));
  std::vector<SolveJob> jobs;
  fct_status s = batch_setup(B, plans, samples, coeffs, team_blocks, Bt->dreps, &jobs, &Bt->G, &Bt->teams, &Bt->smem);
  if (s != FCT_OK) return fail_free(s);
  e = cudaMemcpy(Bt->djobs, jobs.data(), sizeof(SolveJob) * B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail_free(cuda_fail(e, "fct_batch_create"));
  Bt->B = B;
  Bt->block_threads = plans[0]->block_threads;
  Bt->device = plans[0]->device;
  Bt->tns = timeout_ns(plans[0]);
  *out = Bt;
  return FCT_OK;
}

fct_status fct_batch_launch(fct_batch Bt, void* stream) {
  if (!Bt) return fail(FCT_ERR_INVALID_ARG, "NULL batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the whole launch state starts from zero (queue head, error flag, team
  // barriers), also after an abandoned launch
  FCT_CUDA(cudaMemsetAsync(Bt->ls, 0, sizeof(LaunchState), st));
  SolveArgs a{};
  a.jobs = Bt->djobs;
  a.njobs = Bt->B;
  a.team_blocks = Bt->G;
  a.ls = Bt->ls;
  a.timeout_ns = Bt->tns;
  a.smem_bytes = Bt->smem;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(Bt->teams * Bt->G);
  cfg.blockDim = dim3(Bt->block_threads);
  cfg.dynamicSmemBytes = static_cast<size_t>(Bt->smem);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* kargs[] = {&a};
  FCT_CUDA(cudaLaunchKernelExC(&cfg, solve_kernel_for(Bt->block_threads), kargs));
  return FCT_OK;
}

fct_status fct_batch_reports(fct_batch Bt, void* stream, fct_report* reps) {
  if (!Bt || !reps) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int err = 0;
  FCT_CUDA(cudaMemcpyAsync(reps, Bt->dreps, sizeof(fct_report) * Bt->B, cudaMemcpyDeviceToHost, st));
  FCT_CUDA(cudaMemcpyAsync(&err, &Bt->ls->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FCT_CUDA(cudaStreamSynchronize(st));
  if (err != 0) {
    for (int i = 0; i < Bt->B; ++i) reps[i].status = err;
    return fail(static_cast<fct_status>(err), "device-side wait expired in the solver");
  }
  fct_status worst = FCT_OK;
  for (int i = 0; i < Bt->B; ++i)
    if (reps[i].status != FCT_OK && worst == FCT_OK) worst = static_cast<fct_status>(reps[i].status);
  if (worst != FCT_OK) return fail(worst, std::string("solver finished with ") + fct_status_string(worst));
  return FCT_OK;
}

fct_status fct_batch_destroy(fct_batch Bt) {
  if (!Bt) return FCT_OK;
  cudaDeviceSynchronize();
  if (Bt->djobs) cudaFree(Bt->djobs);
  if (Bt->ls) cudaFree(Bt->ls);
  delete Bt;
  return FCT_OK;
}

fct_status fct_destroy(fct_plan P) {
  if (!P) return FCT_OK;
  cudaDeviceSynchronize();
  if (P->d_params) cudaFree(P->d_params);
  if (P->d_stage_in) cudaFree(P->d_stage_in);
  if (P->d_stage_out) cudaFree(P->d_stage_out);
  if (P->djobs) cudaFree(P->djobs);
  if (P->d_hist_block) cudaFree(P->d_hist_block);
  if (P->d_stage_rhs_x) cudaFree(P->d_stage_rhs_x);
  if (P->wmem) cudaFree(P->wmem);
  P->tables.reset();  // frees the table allocation with its last user
  delete P;
  return FCT_OK;
}

fct_status fct_plan_clone(fct_plan* out, fct_plan src) {
  if (!out || !src) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  auto* C = new fct_plan_s();
  C->device = src->device;
  C->opt = src->opt;
  C->H = src->H;
  C->D = src->D;
  C->K = src->K;
  C->N = src->N;
  C->M = src->M;
  C->R = src->R;
  C->dmax = src->dmax;
  C->sizes = src->sizes;
  C->tables = src->tables;
  C->dmem = src->dmem;
  C->dbytes = src->dbytes;
  C->hp = src->hp;
  C->d_sizes = src->d_sizes;
  C->d_offsets = src->d_offsets;
  C->d_node_off = src->d_node_off;
  C->d_node_pos = src->d_node_pos;
  C->d_support = src->d_support;
  C->d_ttab = src->d_ttab;
  C->d_ichunks = src->d_ichunks;
  C->d_emats = src->d_emats;
  C->block_threads = src->block_threads;
  C->grid_blocks = src->grid_blocks;
  C->max_coresident = src->max_coresident;
  C->blocks_per_sm = src->blocks_per_sm;
  C->smem_bytes = src->smem_bytes;
  C->stage_values = src->stage_values;
  C->kernel_kind = src->kernel_kind;
  C->smem_cap = src->smem_cap;
  C->ru_first = src->ru_first;
  C->rowptr_h = src->rowptr_h;
  C->w_rowptr_h = src->w_rowptr_h;
  C->tc = src->tc;
  C->tc_dev = src->tc_dev;
  if (C->tc) {
    auto wk = std::make_shared<TcWork>();
    const fct_status ts = tc_alloc_work(*C->tc, wk.get());
    if (ts != FCT_OK) {
      delete C;
      return ts;
    }
    C->tc_work = wk;
  }
  // its own workspace, DevPlan copy, launch state and report
  DevPlan& hp = C->hp;
  const size_t M = static_cast<size_t>(std::max<int64_t>(C->M, 1)), R = static_cast<size_t>(C->R),
               N = static_cast<size_t>(C->N);
  struct Piece {
    void** dst;
    size_t bytes;
  };
  std::vector<Piece> pieces = {
      {reinterpret_cast<void**>(&C->dp), sizeof(DevPlan)},
      {reinterpret_cast<void**>(&C->ls), sizeof(LaunchState)},
      {reinterpret_cast<void**>(&C->drep), sizeof(fct_report)},
      {reinterpret_cast<void**>(&hp.y0), sizeof(double) * M},
      {reinterpret_cast<void**>(&hp.y1), sizeof(double) * M},
      {reinterpret_cast<void**>(&hp.b), sizeof(double) * R},
      {reinterpret_cast<void**>(&hp.rres), sizeof(double) * R},
      {reinterpret_cast<void**>(&hp.q), sizeof(double) * R},
      {reinterpret_cast<void**>(&hp.sp), sizeof(double2) * N},
      {reinterpret_cast<void**>(&hp.part_r), sizeof(double) * hp.n_row_units},
      {reinterpret_cast<void**>(&hp.part_c), sizeof(double) * hp.n_coef_chunks},
      {reinterpret_cast<void**>(&hp.q32), sizeof(float) * R},
      {reinterpret_cast<void**>(&hp.sp32), sizeof(float2) * N},
      {reinterpret_cast<void**>(&hp.dx32), sizeof(float) * N},
      {reinterpret_cast<void**>(&hp.wv), sizeof(float) * (hp.n_w_units > 0 ? 6 * N : 1)},
      {reinterpret_cast<void**>(&hp.pw64), sizeof(double2) * 2 * std::max(hp.n_w_units, 1)},
  };
  size_t total = 0;
  for (auto& pc : pieces) total += align256(std::max<size_t>(pc.bytes, 1));
  cudaError_t e = cudaMalloc(&C->wmem, total);
  if (e != cudaSuccess) {
    delete C;
    return cuda_fail(e, "cudaMalloc(plan clone)");
  }
  size_t off = 0;
  for (auto& pc : pieces) {
    *pc.dst = C->wmem + off;
    off += align256(std::max<size_t>(pc.bytes, 1));
  }
  e = cudaMemset(C->ls, 0, sizeof(LaunchState));
  if (e == cudaSuccess) e = cudaMemcpy(C->dp, &hp, sizeof(DevPlan), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(C->wmem);
    delete C;
    return cuda_fail(e, "plan clone upload");
  }
  *out = C;
  return FCT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free execute (fct_execute_noalloc)
//
// Some callers cannot allocate device memory when they solve: code running
// under a memory policy that forbids cudaMalloc after start-up (real-time
// loops, fixed memory pools, a host runtime that owns all device memory), or
// code inside a region where an allocation would be unsafe.  They build their
// plans ahead of time and run them through this entry point, whose solver
// workspace lives in the fixed array below instead of in the plan.  The plan
// still provides its read-only tables; nothing is allocated or freed here.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;  // 32 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kNoallocMaxDevices = 64;
void* g_noalloc_addr[kNoallocMaxDevices] = {};  // device address of the array, per device
std::mutex g_noalloc_mu;

// Writes the call's DevPlan into the array from a kernel argument, so no host
// buffer has to outlive the call.
__global__ void noalloc_put_plan_kernel(DevPlan* dst, const DevPlan src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = src;
}

// Layout of the workspace inside the array (256-byte aligned pieces).
struct NoallocLayout {
  size_t devplan, report, ls, y0, y1, b, rres, q, sp, part_r, part_c, q32, sp32, dx32, wv, pw64, total;
};

NoallocLayout noalloc_layout(const fct_plan P) {
  NoallocLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += align256(std::max<size_t>(bytes, 1));
    return at;
  };
  const size_t M = static_cast<size_t>(std::max<int64_t>(P->M, 1)), R = static_cast<size_t>(P->R),
               N = static_cast<size_t>(P->N);
  L.devplan = take(sizeof(DevPlan));
  L.report = take(sizeof(fct_report));
  L.ls = take(sizeof(LaunchState));
  L.y0 = take(sizeof(double) * M);
  L.y1 = take(sizeof(double) * M);
  L.b = take(sizeof(double) * R);
  L.rres = take(sizeof(double) * R);
  L.q = take(sizeof(double) * R);
  L.sp = take(sizeof(double2) * N);
  L.part_r = take(sizeof(double) * P->hp.n_row_units);
  L.part_c = take(sizeof(double) * P->hp.n_coef_chunks);
  L.q32 = take(sizeof(float) * R);
  L.sp32 = take(sizeof(float2) * N);
  L.dx32 = take(sizeof(float) * N);
  L.wv = take(sizeof(float) * (P->hp.n_w_units > 0 ? 6 * N : 1));
  L.pw64 = take(sizeof(double2) * 2 * std::max(P->hp.n_w_units, 1));
  L.total = off;
  return L;
}

}  // namespace

extern "C" fct_status fct_execute_noalloc(fct_plan P, const double* samples, double* coeffs, void* stream,
                                          fct_report* rep) {
  if (!P || !samples || !coeffs) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  const NoallocLayout L = noalloc_layout(P);
  if (L.total > kNoallocScratchBytes)
    return fail(FCT_ERR_INVALID_ARG, "plan needs " + std::to_string(L.total) +
                                         " bytes of solver workspace; fct_execute_noalloc holds at most " +
                                         std::to_string(kNoallocScratchBytes) + " bytes (use fct_execute)");
  int dev = 0;
  FCT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(FCT_ERR_INVALID_ARG, "device index out of range");
  if (dev != P->device) return fail(FCT_ERR_INVALID_ARG, "the current device is not the plan's device");
  void* base = nullptr;
  {
    // First call on this device: look up the array's device address (the host
    // symbol is only a stand-in and must not be handed to a kernel).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  char* b = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The plan's tables with this array's workspace.
  DevPlan hp = P->hp;
  hp.y0 = reinterpret_cast<double*>(b + L.y0);
  hp.y1 = reinterpret_cast<double*>(b + L.y1);
  hp.b = reinterpret_cast<double*>(b + L.b);
  hp.rres = reinterpret_cast<double*>(b + L.rres);
  hp.q = reinterpret_cast<double*>(b + L.q);
  hp.sp = reinterpret_cast<double2*>(b + L.sp);
  hp.part_r = reinterpret_cast<double*>(b + L.part_r);
  hp.part_c = reinterpret_cast<double*>(b + L.part_c);
  hp.q32 = reinterpret_cast<float*>(b + L.q32);
  hp.sp32 = reinterpret_cast<float2*>(b + L.sp32);
  hp.dx32 = reinterpret_cast<float*>(b + L.dx32);
  hp.wv = reinterpret_cast<float*>(b + L.wv);
  hp.pw64 = reinterpret_cast<double2*>(b + L.pw64);
  DevPlan* dplan = reinterpret_cast<DevPlan*>(b + L.devplan);
  fct_report* drep = reinterpret_cast<fct_report*>(b + L.report);
  LaunchState* ls = reinterpret_cast<LaunchState*>(b + L.ls);
  // The array keeps the previous call's contents: the launch header and the
  // team's barrier counters must start at zero.
  FCT_CUDA(cudaMemsetAsync(ls, 0, offsetof(LaunchState, team_job), st));
  FCT_CUDA(cudaMemsetAsync(&ls->bars[0], 0, sizeof(TeamBarrier), st));
  noalloc_put_plan_kernel<<<1, 32, 0, st>>>(dplan, hp);
  FCT_CUDA(cudaGetLastError());
  SolveArgs a{};
  a.single = make_job(P, samples, coeffs, drep);
  a.single.plan = dplan;
  a.jobs = nullptr;
  a.njobs = 1;
  a.team_blocks = P->grid_blocks;
  a.ls = ls;
  a.timeout_ns = timeout_ns(P);
  a.smem_bytes = P->smem_bytes;
  void* kargs[] = {&a};
  FCT_CUDA(cudaLaunchCooperativeKernel(solve_kernel_for(P->block_threads), dim3(P->grid_blocks),
                                       dim3(P->block_threads), kargs, static_cast<size_t>(a.smem_bytes), st));
  if (!rep) return FCT_OK;
  FCT_CUDA(cudaMemcpyAsync(rep, drep, sizeof(fct_report), cudaMemcpyDeviceToHost, st));
  int err = 0;
  FCT_CUDA(cudaMemcpyAsync(&err, &ls->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  FCT_CUDA(cudaStreamSynchronize(st));
  if (err != 0) {
    rep->status = err;
    return fail(static_cast<fct_status>(err), "device-side wait expired in the solver");
  }
  if (rep->status != FCT_OK)
    return fail(static_cast<fct_status>(rep->status),
                std::string("solver finished with ") + fct_status_string(rep->status));
  return FCT_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: a team barrier that cannot complete (one block launched, two
// expected) must give up after the time limit and report FCT_ERR_TIMEOUT,
// leaving the context usable.  No fault, trap or unbounded wait is involved.
// ---------------------------------------------------------------------------
__global__ void wait_selftest_kernel(LaunchState* ls, unsigned long long timeout_ns) {
  Team tm;
  tm.G = 2;  // a partner block that is never launched
  tm.rank = 0;
  tm.epoch = 0;
  tm.bar = &ls->bars[0];
  tm.err = &ls->err;
  tm.timeout_ns = timeout_ns;
  team_sync(tm);
}

extern "C" fct_status fct_selftest_wait_timeout(double timeout_s, int* status_out, double* elapsed_s) {
  if (!status_out || !(timeout_s > 0.0) || timeout_s > 10.0)
    return fail(FCT_ERR_INVALID_ARG, "timeout_s must be in (0, 10]");
  LaunchState* ls = nullptr;
  FCT_CUDA(cudaMalloc(&ls, sizeof(LaunchState)));
  cudaError_t e = cudaMemset(ls, 0, sizeof(LaunchState));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32>>>(ls, static_cast<unsigned long long>(timeout_s * 1e9));
    e = cudaGetLastError();
  }
  cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, &ls->err, sizeof(int), cudaMemcpyDeviceToHost);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(ls);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  *status_out = err;
  if (elapsed_s) *elapsed_s = ms / 1e3;
  return FCT_OK;
}

// ---------------------------------------------------------------------------
// Synchronisation floor: the team barrier alone, `rounds` times over `blocks`
// co-resident blocks (no work between barriers), so that a transform's time
// per CG iteration can be set against two barrier crossings.
// ---------------------------------------------------------------------------
__global__ void barrier_probe_kernel(LaunchState* ls, int rounds, unsigned long long timeout_ns) {
  Team tm;
  tm.G = static_cast<int>(gridDim.x);
  tm.rank = static_cast<int>(blockIdx.x);
  tm.epoch = 0;
  tm.bar = &ls->bars[0];
  tm.err = &ls->err;
  tm.timeout_ns = timeout_ns;
  for (int r = 0; r < rounds; ++r)
    if (!team_sync(tm)) return;
  team_exit(tm);
}

extern "C" fct_status fct_measure_team_barrier(int blocks, int block_threads, int rounds, double* us_per_barrier) {
  if (!us_per_barrier || rounds < 1 || rounds > 1000000 || blocks < 1 ||
      (block_threads != 128 && block_threads != 256 && block_threads != 512))
    return fail(FCT_ERR_INVALID_ARG, "need blocks >= 1, block_threads 128/256/512, rounds in [1, 1e6]");
  int dev = 0, nsm = 0, per_sm = 0;
  FCT_CUDA(cudaGetDevice(&dev));
  FCT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  FCT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_probe_kernel, block_threads, 0));
  if (blocks > per_sm * nsm) return fail(FCT_ERR_INVALID_ARG, "more blocks than can be co-resident");
  LaunchState* ls = nullptr;
  FCT_CUDA(cudaMalloc(&ls, sizeof(LaunchState)));
  cudaError_t e = cudaMemset(ls, 0, sizeof(LaunchState));
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  unsigned long long tns = 4000000000ull;
  void* kargs[] = {&ls, &rounds, &tns};
  if (e == cudaSuccess) e = cudaEventRecord(a);
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(barrier_probe_kernel), dim3(blocks),
                                    dim3(block_threads), kargs, 0, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int err = 0;
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaMemcpy(&err, &ls->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(ls);
  if (e != cudaSuccess) return cuda_fail(e, "team barrier probe");
  if (err != 0) return fail(static_cast<fct_status>(err), "team barrier probe: a wait expired");
  *us_per_barrier = 1e3 * static_cast<double>(ms) / rounds;
  return FCT_OK;
}

// ---------------------------------------------------------------------------
// Serving (continuous batching): a persistent launch whose teams take jobs
// from a ring in host-mapped memory as they are published; a job submitted
// while others run is picked up by the next team that frees up.  When no job
// arrives for idle_timeout the launch ends; the next submit (or a wait on an
// unclaimed job) launches it again.
// ---------------------------------------------------------------------------
struct fct_server_s {
  int device = 0;
  int block_threads = 256;
  int team_blocks = 0;
  int teams = 0;
  int smem_bytes = 0;
  unsigned long long idle_ns = 0;
  unsigned long long timeout_ns = 4000000000ull;
  ServerRing* h_ring = nullptr;  // host view of the mapped ring
  ServerRing* d_ring = nullptr;  // device view
  LaunchState* ls = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done_ev = nullptr;
  bool launched = false;
  unsigned long long next = 0;
  std::mutex mu;
};

namespace {

fct_status server_ensure_running(fct_server S) {
  const int derr = __atomic_load_n(&S->h_ring->err, __ATOMIC_ACQUIRE);
  if (derr != 0)
    return fail(static_cast<fct_status>(derr), "the serving launch abandoned its jobs after a device-side error");
  if (S->launched && cudaEventQuery(S->done_ev) == cudaErrorNotReady) return FCT_OK;
  if (S->launched) {
    int err = 0;
    FCT_CUDA(cudaMemcpy(&err, &S->ls->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err != 0) return fail(static_cast<fct_status>(err), "serving launch ended with a device-side error");
  }
  // busy, exiting and last_ns start from zero; queue_head keeps its place in the ring
  FCT_CUDA(cudaMemsetAsync(&S->ls->busy, 0, 2 * sizeof(int) + sizeof(unsigned long long), S->stream));
  SolveArgs a{};
  a.jobs = nullptr;
  a.njobs = 0;
  a.team_blocks = S->team_blocks;
  a.ls = S->ls;
  a.timeout_ns = S->timeout_ns;
  a.smem_bytes = S->smem_bytes;
  a.ring = S->d_ring;
  a.idle_ns = S->idle_ns;
  void* kargs[] = {&a};
  FCT_CUDA(cudaLaunchCooperativeKernel(solve_kernel_for(S->block_threads), dim3(S->teams * S->team_blocks),
                                       dim3(S->block_threads), kargs, static_cast<size_t>(S->smem_bytes), S->stream));
  FCT_CUDA(cudaEventRecord(S->done_ev, S->stream));
  S->launched = true;
  return FCT_OK;
}

}  // namespace

extern "C" {

fct_status fct_server_create(fct_server* out, int block_threads, int team_blocks, int teams, double idle_timeout_s) {
  if (!out) return fail(FCT_ERR_INVALID_ARG, "out must not be NULL");
  *out = nullptr;
  if (block_threads == 0) block_threads = 256;
  if (block_threads != 128 && block_threads != 256 && block_threads != 512)
    return fail(FCT_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
  if (!(idle_timeout_s > 0.0) || idle_timeout_s > 1.0) return fail(FCT_ERR_INVALID_ARG, "idle_timeout_s must be in (0, 1]");
  int dev = 0, nsm = 0, per_sm = 0, cap = 0;
  FCT_CUDA(cudaGetDevice(&dev));
  FCT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaDeviceProp prop;
  FCT_CUDA(cudaGetDeviceProperties(&prop, dev));
  const fct_status cs = solver_smem_cap(block_threads, prop, &cap, &per_sm);
  if (cs != FCT_OK) return cs;
  if (cap < coef_combine_bytes(block_threads)) return fail(FCT_ERR_CUDA, "no shared memory for the solver");
  const int coresident = per_sm * nsm;
  if (team_blocks <= 0) team_blocks = 16;
  team_blocks = std::min(team_blocks, coresident);
  const int max_teams = std::min(coresident / team_blocks, kMaxTeams);
  if (teams <= 0 || teams > max_teams) teams = max_teams;
  auto* S = new fct_server_s();
  S->device = dev;
  S->block_threads = block_threads;
  S->team_blocks = team_blocks;
  S->teams = teams;
  S->smem_bytes = cap;
  S->idle_ns = static_cast<unsigned long long>(idle_timeout_s * 1e9);
  cudaError_t e = cudaHostAlloc(&S->h_ring, sizeof(ServerRing), cudaHostAllocMapped | cudaHostAllocPortable);
  if (e == cudaSuccess) {
    std::memset(S->h_ring, 0, sizeof(ServerRing));
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->d_ring), S->h_ring, 0);
  }
  if (e == cudaSuccess) e = cudaMalloc(&S->ls, sizeof(LaunchState));
  if (e == cudaSuccess) e = cudaMemset(S->ls, 0, sizeof(LaunchState));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->done_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (S->h_ring) cudaFreeHost(S->h_ring);
    if (S->ls) cudaFree(S->ls);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return cuda_fail(e, "fct_server_create");
  }
  *out = S;
  return FCT_OK;
}

fct_status fct_server_submit(fct_server S, fct_plan P, const double* samples, double* coeffs, int64_t* ticket) {
  if (!S || !P || !samples || !coeffs || !ticket) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  if (P->block_threads != S->block_threads) return fail(FCT_ERR_INVALID_ARG, "plan block_threads differs from the server's");
  std::lock_guard<std::mutex> lk(S->mu);
  const unsigned long long j = S->next;
  ServerSlot& slot = S->h_ring->slots[j % kRingSize];
  if (j >= static_cast<unsigned long long>(kRingSize) && __atomic_load_n(&slot.done, __ATOMIC_ACQUIRE) == 0)
    return fail(FCT_ERR_OOM, "serving ring full: the job submitted 4096 tickets ago has not finished");
  slot.job = make_job(P, samples, coeffs, &S->d_ring->slots[j % kRingSize].rep);
  std::memset(&slot.rep, 0, sizeof(slot.rep));
  __atomic_store_n(&slot.done, 0, __ATOMIC_RELAXED);
  __atomic_store_n(&S->h_ring->tail, j + 1, __ATOMIC_RELEASE);  // publishes the slot
  S->next = j + 1;
  *ticket = static_cast<int64_t>(j);
  return server_ensure_running(S);
}

fct_status fct_server_poll(fct_server S, int64_t ticket, int* done, fct_report* rep) {
  if (!S || !done || ticket < 0) return fail(FCT_ERR_INVALID_ARG, "bad argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (static_cast<unsigned long long>(ticket) >= S->next) return fail(FCT_ERR_INVALID_ARG, "unknown ticket");
  ServerSlot& slot = S->h_ring->slots[ticket % kRingSize];
  *done = __atomic_load_n(&slot.done, __ATOMIC_ACQUIRE);
  if (*done) {
    if (rep) *rep = slot.rep;
    return FCT_OK;
  }
  // not finished: a device-side error published by the running launch ends
  // the wait here (the job will never be solved); otherwise a job published
  // just as the launch went idle is picked up by a new launch
  return server_ensure_running(S);
}

fct_status fct_server_wait(fct_server S, int64_t ticket, double timeout_s, fct_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    int done = 0;
    fct_status st = fct_server_poll(S, ticket, &done, rep);
    if (st != FCT_OK) return st;
    if (done) return rep ? static_cast<fct_status>(rep->status) : FCT_OK;
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > timeout_s) return fail(FCT_ERR_TIMEOUT, "fct_server_wait: job not finished in time");
    std::this_thread::yield();
  }
}

fct_status fct_server_destroy(fct_server S) {
  if (!S) return FCT_OK;
  __atomic_store_n(&S->h_ring->stop, 1, __ATOMIC_RELEASE);
  cudaStreamSynchronize(S->stream);
  cudaEventDestroy(S->done_ev);
  cudaStreamDestroy(S->stream);
  cudaFree(S->ls);
  cudaFreeHost(S->h_ring);
  delete S;
  return FCT_OK;
}

}  // extern "C"


// ---------------------------------------------------------------------------
// Condition estimate for Algorithm 2's test kappa(A) <= kappa0: CG on A^T A is
// the Lanczos process, so its coefficients give the Lanczos tridiagonal T_k
//   T[j][j] = 1/alpha_j + beta_j/alpha_{j-1},  T[j][j+1] = sqrt(beta_{j+1})/alpha_j,
// whose extreme eigenvalues (Ritz values) approach those of A^T A from inside:
// sqrt(lambda_max / lambda_min) is a lower bound on kappa(A) that tightens
// with k.
// ---------------------------------------------------------------------------
namespace {

// number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm)
int sturm_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double e2 = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
    q = (d[i] - x) - (i > 0 ? e2 / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}

void tridiag_extremes(const std::vector<double>& d, const std::vector<double>& e, double* lmin, double* lmax) {
  const size_t k = d.size();
  double lo = d[0], hi = d[0];
  for (size_t i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  double a = lo, b = hi;  // smallest: count(x) >= 1
  for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
    const double m = 0.5 * (a + b);
    if (sturm_below(d, e, m) >= 1) b = m; else a = m;
  }
  *lmin = 0.5 * (a + b);
  a = lo;
  b = hi;  // largest: count(x) >= k
  for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
    const double m = 0.5 * (a + b);
    if (sturm_below(d, e, m) >= static_cast<int>(k)) b = m; else a = m;
  }
  *lmax = 0.5 * (a + b);
}

}  // namespace

extern "C" fct_status fct_plan_condition(fct_plan P, const double* start, double* work, int iterations,
                                         double* kappa, double* lambda_min, double* lambda_max, int* used,
                                         void* stream) {
  if (!P || !start || !work || !kappa) return fail(FCT_ERR_INVALID_ARG, "NULL argument");
  if (iterations < 2 || iterations > 100000) return fail(FCT_ERR_INVALID_ARG, "iterations must be in [2, 100000]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (P->hist_cap < iterations) {
    if (P->d_hist_block) {
      FCT_CUDA(cudaStreamSynchronize(st));
      cudaFree(P->d_hist_block);
      P->d_hist_block = nullptr;
      P->hist_cap = 0;
    }
    FCT_CUDA(cudaMalloc(&P->d_hist_block, align256(sizeof(DevPlan)) + sizeof(double2) * iterations));
    P->hist_cap = iterations;
  }
  DevPlan hp = P->hp;
  hp.s_init = start;
  hp.hist = reinterpret_cast<double2*>(P->d_hist_block + align256(sizeof(DevPlan)));
  hp.hist_cap = iterations;
  DevPlan* dplan = reinterpret_cast<DevPlan*>(P->d_hist_block);
  FCT_CUDA(cudaMemcpyAsync(dplan, &hp, sizeof(DevPlan), cudaMemcpyHostToDevice, st));
  FCT_CUDA(cudaMemsetAsync(hp.hist, 0, sizeof(double2) * iterations, st));
  SolveArgs a{};
  a.single = make_job(P, nullptr, work, P->drep);
  a.single.plan = dplan;
  a.single.precision = FCT_FP64;
  a.single.max_iter = iterations;
  // Stop once the normal residual has fallen by 1e12: the extreme Ritz values
  // have converged by then, and the CG coefficients of a nearly converged
  // iteration carry mostly rounding.
  a.single.tol = 1e-12;
  a.jobs = nullptr;
  a.njobs = 1;
  a.team_blocks = P->grid_blocks;
  a.ls = P->ls;
  a.timeout_ns = timeout_ns(P);
  a.smem_bytes = P->smem_bytes;
  fct_status s = launch_solve(P, a, P->grid_blocks, st);
  if (s != FCT_OK) return s;
  fct_report rep;
  s = read_report(P, P->drep, st, &rep);
  if (s != FCT_OK && s != FCT_ERR_NOCONV) return s;
  std::vector<double2> h(iterations);
  FCT_CUDA(cudaMemcpy(h.data(), hp.hist, sizeof(double2) * iterations, cudaMemcpyDeviceToHost));
  int k = std::min(rep.iterations, iterations);
  for (int j = 0; j < k; ++j)
    if (!(h[j].x > 0.0) || !std::isfinite(h[j].x) || !(h[j].y >= 0.0) || !std::isfinite(h[j].y)) {
      k = j;
      break;
    }
  if (k < 1) return fail(FCT_ERR_INVALID_ARG, "the probe recorded no iteration (zero start vector?)");
  std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
  for (int j = 0; j < k; ++j) {
    const double al = h[j].x;
    d[j] = 1.0 / al + (j > 0 ? h[j].y / h[j - 1].x : 0.0);
    if (j + 1 < k) e[j] = std::sqrt(h[j + 1].y) / al;
  }
  double lmin = 0.0, lmax = 0.0;
  tridiag_extremes(d, e, &lmin, &lmax);
  if (lambda_min) *lambda_min = lmin;
  if (lambda_max) *lambda_max = lmax;
  if (used) *used = k;
  *kappa = lmin > 0.0 ? std::sqrt(lmax / lmin) : INFINITY;
  return FCT_OK;
}
