// Internal structures of the GB300 sparse-FCT library (host plan builder and
// device kernels).  Not part of the public ABI (include/fct.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "fct.h"

namespace fct {

constexpr int kMaxD = 255;
constexpr int kDctChunk = 1024;        // elements of one grid per DCT work unit
constexpr int kMaxTeams = 1024;        // teams per launch (batched execute)
constexpr int kMaxAxis = 4096;         // longest grid axis (points) the direct DCT-I accepts
// Gather lane classes of a row: 1, 2, 4, 8, 16, 32 lanes, or kWideLanes: a row
// longer than kWideRowFactor * 32 lanes * (entries per lane) is gathered by
// every gather warp of a block (one row per unit), the warps' partial sums
// added in warp order.
constexpr int kWideLanes = 64;
constexpr int kWideRowFactor = 16;
constexpr int kLaneClasses = 7;

// Solver row order: ascending key = (class number, 6 - log2(lanes): wide rows
// first, then 32 lanes, ..., 1 lane) above 16 bits that are zero unless the
// plan has at least kRoundsOrderMinEntries table entries (K N); there they
// hold 65535 - load rounds, the rounds being ceil(len / (32 * epl)) capped at
// 65535.  Rows of fewer than 32 lanes take one round by construction, so only
// 32-lane and wide rows move: longest first, so that the rows a block's warps
// take side by side between two block barriers need about as many rounds.
// Smaller plans keep the class order alone: their blocks stage their units in
// shared memory in unit order, and a block whose first unit holds all the
// longest rows would stage fewer of its units than the others.  Both row
// builders sort stably by this key (equal keys keep ascending bin order).
// lanes = lanes_for(len, epl).
constexpr int64_t kRoundsOrderMinEntries = int64_t(1) << 23;
#ifdef __CUDACC__
__host__ __device__
#endif
inline int32_t row_order_key(int64_t len, int lanes, int epl, bool by_rounds) {
  int cls = 0;
  while ((1 << cls) < lanes) ++cls;
  const int64_t per = 32 * static_cast<int64_t>(epl);
  int64_t rounds = (len + per - 1) / per;
  if (rounds > 65535) rounds = 65535;
  return static_cast<int32_t>(((kLaneClasses - 1 - cls) << 16) | (by_rounds ? 65535 - rounds : 0));
}
constexpr int kRowOrderKeyBits = 19;  // class (3 bits) above 16 bits of rounds

// One DCT-I work unit: a contiguous element range of one grid tensor in one
// axis pass.  Output element e (within the grid) is
//   out[e] = sum_j C[k][j] * in[e - k*stride + j*stride],  k = (e/stride) % n.
struct DctChunk {
  int64_t base;            // grid's first sample in samples / y0 / y1
  int32_t start, count;    // element range within the grid tensor (fibre range when fibres = 1)
  int32_t n, stride;       // axis length (1 = identity copy) and its stride
  int32_t mat;             // offset of the n x n matrix in dct_mats
  int8_t in_sel, out_sel;  // 0 = caller samples, 1 = y0, 2 = y1, 3 = caller samples (output)
  int16_t fibres;          // 1: one thread per fibre computes all n outputs (even/odd split)
};
// Forward DCT passes of axes with kFibreMinN..kFibreMaxN points run one thread
// per fibre, kFibreChunk fibres per work unit, when the pass has at least
// kFibrePassMin fibres over all grids (several waves of GB300 threads).
constexpr int kFibreMinN = 2;
constexpr int kFibreMaxN = 16;
constexpr int kFibreChunk = 512;
constexpr int64_t kFibrePassMin = int64_t{1} << 18;
static_assert(sizeof(DctChunk) == 32, "DctChunk layout");

// Last DCT-I pass of a grid, evaluated only at its nonempty bins (fused with
// the gather of b): b[row] = sum_j C[k][j] * in[rowbase[row] + j*stride].
struct GridFinal {
  int32_t n, stride, mat;
  int32_t in_sel;          // 0 = caller samples, 1 = y0, 2 = y1
};

// ---------------------------------------------------------------------------
// DCT passes on the tensor cores (grids with a long axis).  An axis pass over a
// grid tensor of shape (pre, n, post) is the product Y = C X of the n x n DCT
// matrix with the n x (pre post) matrix of the tensor's fibres.  Both factors
// are split into kTcSlices slices of 8-bit signed digits (base 128, balanced)
// below a per-row (C) and per-column (X) power of two, so every slice is
// exact in BF16; the products of slice pairs with digit sum g (36 products)
// accumulate exactly in FP32 on the tensor cores (|sum| < 2^24 for n <= 1024)
// and the kTcSlices sums are combined in integers, then converted to FP64 once
// per output: results agree with an FP64 product to about 1e-16 relative to
// sum |C||X|.  M tile 128 rows of C, N tile 64 fibres, K step 16.
// ---------------------------------------------------------------------------
constexpr int kTcSlices = 8;
constexpr int kTcM = 128, kTcN = 64, kTcK = 16;
constexpr int kTcATile = kTcM * kTcK * 2;             // bytes of one A slice of one K step
constexpr int kTcBTile = kTcN * kTcK * 2;             // bytes of one B slice of one K step
constexpr int kTcAStep = kTcSlices * kTcATile;        // 32 KB: all A slices of one K step
constexpr int kTcBStep = kTcSlices * kTcBTile;        // 16 KB
constexpr int kTcStageBytes = kTcAStep + kTcBStep;    // one pipeline stage in shared memory
constexpr int kTcStages = 4;
constexpr int kTcMinAxis = 64;                        // auto: grids whose longest axis has >= 64 points
constexpr int kTcMaxAxis = 1024;                      // exact FP32 accumulation holds up to here
constexpr int kTcNonFinite = -100000;                 // column exponent of a fibre holding NaN / Inf

// One tensor-core pass over one grid.
struct TcGridPass {
  int64_t base;      // the grid's first element in samples / y0 / y1
  int64_t a_off;     // byte offset of the A slices of this axis length
  int64_t b_off;     // byte offset of this pass's B slices in the B workspace
  int32_t n, post;   // axis length and stride: the tensor is (pre, n, post)
  int32_t ncols;     // pre * post fibres
  int32_t ksteps;    // ceil(n / 16)
  int32_t mtiles, ntiles;
  int32_t e_off;     // first row exponent of this axis length
  int32_t f_off;     // first column exponent of this pass in the exponent workspace
  int8_t in_sel, out_sel;  // 0 = caller samples, 1 = y0, 2 = y1
  int16_t pad0;
  int32_t pad1;
};
static_assert(sizeof(TcGridPass) == 64, "TcGridPass layout");

// Host description of a plan's tensor-core DCT (empty when no grid uses it).
struct TcHost {
  std::vector<char> grid_tc;              // [K] 1 = the grid's DCT runs on the tensor cores
  int npass = 0;                          // tensor-core passes (most active axes of a tensor-core grid)
  std::vector<TcGridPass> gp;             // all passes, pass-major
  std::vector<int32_t> gp_off;            // [npass + 1]
  std::vector<int32_t> split_tasks;       // pairs {gp, ntile}
  std::vector<int32_t> split_off;         // [npass + 1] in pairs
  std::vector<int32_t> gemm_tasks;        // quads {gp, mtile, ntile, 0}
  std::vector<int32_t> gemm_off;          // [npass + 1] in quads
  std::vector<uint16_t> a_bits;           // BF16 bits of every A slice
  std::vector<int32_t> a_exp;             // row exponents
  int64_t b_bytes = 0;                    // B workspace (largest pass)
  int32_t max_ksteps = 0;                 // most K steps of any pass
  int64_t f_count = 0;                    // column-exponent workspace (largest pass)
  // the solver's DCT for plans run with the tensor-core passes: passes of the
  // grids left to the FP64 units, and a last pass that reads the finished
  // transform of every tensor-core grid (identity)
  int npass_fp64 = 0;
  std::vector<int32_t> pass_chunk_off;
  std::vector<DctChunk> dct_chunks;
  std::vector<GridFinal> gfinal;
  bool empty() const { return npass == 0; }
};

// Plans with at least this many grids take the grid-split A^T q gather
// unless fct_options.coef_split says otherwise.
constexpr int kCoefSplitMinGrids = 64;
// Shared memory of the grid-split gather's partial sums, at the start of a
// block's dynamic shared memory: two buffers of (gather warps x 32) doubles.
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int coef_combine_bytes(int block_threads) { return 2 * (block_threads / 32 - 1) * 32 * 8; }

// Everything the solver kernel needs about one plan; lives in device memory.
struct DevPlan {
  int32_t N, R, K, D;
  int64_t M;
  int32_t npass;             // full DCT axis passes (every grid's last pass is fused into b)
  int32_t n_row_units;       // A p gather units (adaptive lanes per row)
  int32_t n_rowel_chunks;    // elementwise units over rows: ceil(R / workers)
  int32_t n_coef_chunks;     // A^T q gather units: ceil(N / coefs_per_chunk)
  int32_t coefs_per_chunk;   // = workers / coef_lanes
  int32_t coef_lanes;        // threads per coefficient in the A^T q gather
  int32_t coef_split;        // 1: grid-split A^T q gather (32 coefficients per chunk, warps over grids)
  int32_t workers;           // gather threads per block (block threads - 32)
  int32_t mats_smem;         // doubles of DCT matrices to stage in shared memory (0 = read global)
  int32_t n_mats;            // doubles in dct_mats
  int32_t n_wide_units;      // leading row units that are wide rows (they sort first)
  // DCT
  const int32_t* pass_chunk_off;  // [npass + 1]
  const DctChunk* dct_chunks;
  const double* dct_mats;
  const GridFinal* gfinal;   // [K]
  const int32_t* rowbase;    // [R] first input element of the row's last-pass fibre
  const int32_t* rowk;       // [R] output index k of the row's bin on the last axis
  const int32_t* rowgrid;    // [R] grid of the row
  // alias tables
  const int32_t* ru_first;   // [n_row_units] first row of each A p unit
  const int32_t* ru_lanes;   // [n_row_units] lanes per row in the unit (power of 2 <= 32)
  const int32_t* rowptr;     // [R+1]  CSR by bin, rows sorted by descending length
  const int32_t* col;        // [K*N]  column of each CSR entry (m ascending in a bin)
  const double* wcsr;        // [K*N]  entry value, CSR order
  const float* wcsr32;       // [K*N]
  const int32_t* crow;       // [K*N]  crow[l*N + m] = row of column m on grid l
  const double* wcm;         // [K*N]  entry value, coefficient-major order
  const float* wcm32;        // [K*N]
  // FP64 workspace
  double* y0;                // [M]
  double* y1;                // [M]
  double* b;                 // [R]
  double* rres;              // [R] FP64 residual b - A x (mixed path sweeps)
  double* q;                 // [R]
  double2* sp;               // [N] {s, p} interleaved: one 16-byte gather per entry
  double* part_r;            // [n_row_units]    FP64 per-unit partial sums (|q|^2 and the set-up phases)
  double* part_c;            // [n_coef_chunks]  (|s|^2 and the refinement sweeps)
  // FP32 workspace of the mixed path
  float* q32;                // [R]
  float2* sp32;              // [N] {s, p} of the inner FP32 solve
  float* dx32;               // [N]
  // normal matrix W = A^T A of the mixed path's inner solve (n_w_units = 0:
  // not built; the inner solve then applies A and A^T in two phases)
  const int32_t* wrowptr;    // [N+1]
  const int32_t* wcol;       // [nnz_w]
  const float* wval;         // [nnz_w]
  int32_t n_w_units;         // units of w_rows_per_unit consecutive rows
  int32_t w_lanes;           // threads per row of W
  int32_t w_rows_per_unit;   // = workers / w_lanes
  int32_t pad_w;
  float* wv;                 // [6N] w (two buffers), r, p, s, z of the pipelined CG
  double2* pw64;             // [2 * n_w_units] FP64 partials (r.r, w.r), two buffers
  // condition estimate: when set, the FP64 solve starts from s = s_init (no
  // DCT, no b) and block 0 records (alpha_k, beta_k) of every CG iteration,
  // the Lanczos coefficients of A^T A for the start vector s_init
  const double* s_init;      // [N] or nullptr
  double2* hist;             // [hist_cap] (alpha_k, beta_k) or nullptr
  int32_t hist_cap;
  int32_t npass_tc;          // jobs with kJobTcDct: FP64 passes left after the tensor-core passes
  // DCT of jobs with kJobTcDct (the tensor-core grids are already transformed
  // in y0 / y1): their pass lists, last passes and last-pass rows
  const int32_t* pass_chunk_off_tc;
  const DctChunk* dct_chunks_tc;
  const GridFinal* gfinal_tc;
  const int32_t* rowbase_tc;
  const int32_t* rowk_tc;
};

// One transform of a launch.
struct SolveJob {
  const DevPlan* plan;       // device pointer
  const double* samples;     // device [M]
  double* coeffs;            // device [N]
  fct_report* report;        // device, one per job
  int32_t precision;
  int32_t max_iter;
  int32_t max_refine;
  int32_t flags;             // kJobPrepareOnly: stop after b and s = A^T b (the DCT stage alone);
                             // kJobTcDct: the tensor-core grids' DCT is done (y0 / y1)
  double tol;
  double inner_tol;
};
constexpr int32_t kJobPrepareOnly = 1;
constexpr int32_t kJobTcDct = 2;

// Barrier of one team: a monotonic arrival counter (target = G x barrier
// number) and an exit counter that lets the last block reset it.
struct TeamBarrier {
  unsigned int count;
  unsigned int pad0[31];
  unsigned int exits;
  unsigned int pad1[31];
};

// Per-launch device state (zeroed before every launch; a serving launch keeps
// queue_head and resets busy / exiting / last_ns).
struct LaunchState {
  unsigned int queue_head;
  int err;
  // serving mode: teams stay while any job runs or ran recently, and once one
  // team decides the whole launch is idle, no team claims another job
  int busy;                   // jobs in progress
  int exiting;                // set by the first team that leaves
  unsigned long long last_ns; // %globaltimer at the last job claim or finish
  int pad[26];
  int team_job[kMaxTeams];
  TeamBarrier bars[kMaxTeams];
};
static_assert(offsetof(LaunchState, exiting) == offsetof(LaunchState, busy) + 4 &&
                  offsetof(LaunchState, last_ns) == offsetof(LaunchState, busy) + 8 &&
                  offsetof(LaunchState, team_job) == 128,
              "LaunchState layout");

// Serving ring in host-mapped memory: the host publishes jobs (slot then
// tail, release), team leaders claim them through LaunchState::queue_head,
// and each finished job gets its report and done flag (system-scope release).
constexpr int kRingSize = 4096;

struct ServerSlot {
  SolveJob job;
  fct_report rep;
  int done;
  int pad[15];
};

struct ServerRing {
  unsigned long long tail;  // jobs published so far (monotonic)
  int stop;                 // host asks the serving kernel to leave
  int err;                  // device: the launch's error code once a team abandoned its job
  int pad[12];
  ServerSlot slots[kRingSize];
};

// Host-side alias tables of a plan (also exported by fct_alias_tables_host).
// Rows are numbered grid by grid, nonempty bins in ascending bin order;
// device_row_order() renumbers them for the solver.
struct HostTables {
  int D = 0, K = 0;
  int64_t N = 0, M = 0, R = 0;
  std::vector<int64_t> offsets;        // [K+1] sample offsets
  std::vector<int32_t> bin;            // [K*N] full-grid bin of m on grid l
  std::vector<int32_t> crow;           // [K*N] global compressed row
  std::vector<double> weight;          // [K*N] coefficient-major entries
  std::vector<int32_t> rowptr;         // [R+1]
  std::vector<int32_t> col;            // [K*N]
  std::vector<double> wcsr;            // [K*N]
  std::vector<int32_t> rowsrc;         // [R] global index into y0 (offset + bin)
  std::vector<int32_t> rowgrid;        // [R] grid of each row
  std::vector<int32_t> row_off;        // [K+1] first row of each grid
  // DCT: full passes (all but each grid's last), then the fused last pass
  int npass = 0;
  std::vector<int32_t> pass_chunk_off; // [npass+1]
  std::vector<DctChunk> dct_chunks;
  std::vector<double> dct_mats;
  std::vector<GridFinal> gfinal;       // [K]
  // inverse transform (sampler of polynomials through the bins): evaluation
  // passes over every active axis, y0/y1 ping-pong, the last into the caller's
  // samples (out_sel 3)
  int nipass = 0;
  std::vector<int32_t> ipass_chunk_off;  // [nipass+1]
  std::vector<DctChunk> idct_chunks;
  std::vector<double> eval_mats;         // E[j][k] = T_k(x_j) per distinct axis length
  // sampler geometry: node positions of every grid axis
  std::vector<int32_t> node_off;       // [K*D] offset of grid l axis i in nodes
  std::vector<double> node_pos;
};

// Validates inputs and builds all host tables.  Returns FCT_OK or an error with
// the message in *err.
// with_alias = false leaves the alias tables (bin, crow, weight, CSR, rows)
// empty for build_device_tables to fill.
fct_status build_host_tables(int D, int64_t N, const uint16_t* support, int K,
                             const int32_t* sizes, const double* nodes, int grid_kind, bool with_dct,
                             HostTables* out, std::string* err, bool with_alias = true);

// Alias tables built on the device (fct_plan_device.cu), already in the
// device row order: the same arrays, bit for bit, as build_host_tables +
// device_row_order.  All pointers live in one scratch allocation.
struct DeviceTables {
  void* mem = nullptr;
  int32_t* rowptr = nullptr;   // [R+1]
  int32_t* rowgrid = nullptr;  // [R]
  int32_t* rowbase = nullptr;  // [R] last-pass fibre start of each row (as final_pass_rows)
  int32_t* rowk = nullptr;     // [R] and the row's index along that fibre
  int32_t* col = nullptr;      // [K N] bin-major
  double* wcsr = nullptr;
  float* wcsr32 = nullptr;
  int32_t* crow = nullptr;     // [K N] coefficient-major
  double* wcm = nullptr;
  float* wcm32 = nullptr;
  void* stream = nullptr;      // cudaStream_t of the build: allocation and release are ordered on it
  void release();
  ~DeviceTables() { release(); }
};

// Builds the alias tables of H's plan on the current device (H holds the
// offsets, D, K, N and the DCT set-up from build_host_tables(with_alias =
// false)).  Chooses the entries per lane as the host path does
// (pick_entries_per_lane), fills H->R, H->rowptr and H->rowsrc in the device
// row order, and out->rowbase / out->rowk as final_pass_rows would.
// Every launch, copy, allocation and release of the build is ordered on
// `stream` (a cudaStream_t); the call synchronises that stream only, so a plan
// can be built while other streams (a serving launch) keep the device busy.
fct_status build_device_tables(HostTables* H, const uint16_t* support, const int32_t* sizes, const double* nodes,
                               int grid_kind, int workers, int64_t wave, int fixed_epl, int* epl,
                               DeviceTables* out, void* stream);
// Copies col, wcsr, crow and the coefficient-major values back into H.
fct_status download_device_tables(const DeviceTables& T, HostTables* H);

// Rows per lane class: classes[q][c] counts the rows with 2^c gather lanes
// (c = 6: wide rows) at 2 << q entries per lane.  The entries per lane of a plan: `fixed` if > 0,
// else the fewest of 2, 4, 8 whose row units fit in `wave` blocks, else 8.
void lane_class_counts(const HostTables& H, int64_t classes[3][kLaneClasses]);
int64_t units_from_classes(const int64_t* per_class, int workers);
int pick_entries_per_lane(const int64_t classes[3][kLaneClasses], int workers, int64_t wave, int fixed);

// Gather lanes of a row with len entries: min(32, pow2 >= ceil(len / epl)),
// epl = target entries per lane; kWideLanes for rows longer than
// kWideRowFactor * 32 * epl.
int lanes_for(int32_t len, int epl);

// Renumber the rows of H for the device: stable sort by row_order_key
// (descending gather lane count, then descending load rounds), so that rows
// with equal lane counts are contiguous; equal keys keep their ascending-bin
// order.  Rewrites rowptr, col, wcsr, rowsrc, rowgrid and crow in place.
void device_row_order(HostTables* H, int epl);

// A p gather units for `workers` threads per block: a unit holds
// workers / lanes consecutive rows of equal lane count.
void row_units(const HostTables& H, int workers, int epl, std::vector<int32_t>* first, std::vector<int32_t>* lanes);

// W = A^T A (N x N, CSR, columns ascending, FP64 sums in a fixed order) and
// the bound sum over rows of A of (row length)^2 >= nnz(W), cheap to compute
// before deciding to build W.
int64_t normal_matrix_bound(const HostTables& H);
void normal_matrix(const HostTables& H, std::vector<int32_t>* rowptr, std::vector<int32_t>* col,
                   std::vector<double>* val);

// Per-row inputs of the fused last DCT pass (after device_row_order).
void final_pass_rows(const HostTables& H, std::vector<int32_t>* rowbase, std::vector<int32_t>* rowk);

// The same for the last passes `gfinal` (one per grid), from each row's sample
// index H.rowsrc (the row's grid is found from the sample offsets).
void final_pass_rows_for(const HostTables& H, const std::vector<GridFinal>& gfinal, std::vector<int32_t>* rowbase,
                         std::vector<int32_t>* rowk);

// Tensor-core DCT set-up: mode 0 = auto (grids whose longest active axis has
// at least kTcMinAxis points), 1 = every grid with an active axis, -1 = none;
// grids with an axis longer than kTcMaxAxis stay on the FP64 units.  Fills
// *T (empty when no grid qualifies); H must hold the DCT set-up of
// build_host_tables.  Adds the identity matrix to H->dct_mats if needed.
fct_status build_tc_host(HostTables* H, const int32_t* sizes, int grid_kind, int mode, TcHost* T);

// Device copy of a TcHost (read-only part) and one workspace.
struct TcDevice {
  void* mem = nullptr;
  const TcGridPass* gp = nullptr;
  const int32_t* split_tasks = nullptr;
  const int32_t* gemm_tasks = nullptr;
  const unsigned char* a = nullptr;
  const int32_t* a_exp = nullptr;
  int32_t* pass_chunk_off = nullptr;
  DctChunk* dct_chunks = nullptr;
  GridFinal* gfinal = nullptr;
  int32_t* rowbase = nullptr;
  int32_t* rowk = nullptr;
  ~TcDevice();
};
struct TcWork {
  void* mem = nullptr;
  unsigned char* b = nullptr;
  int32_t* f = nullptr;
  ~TcWork();
};
fct_status tc_upload(const TcHost& T, const std::vector<int32_t>& rowbase, const std::vector<int32_t>& rowk,
                     TcDevice* out);
fct_status tc_alloc_work(const TcHost& T, TcWork* out);
// Runs every tensor-core pass of the plan on `stream`: the finished transforms
// of the tensor-core grids land in y0 / y1 as the solver's kJobTcDct jobs
// expect.  A bounded wait that expires sets *err (the launch's error flag).
fct_status tc_run(const TcHost& T, const TcDevice& D, const TcWork& Wk, const double* samples, double* y0,
                  double* y1, int* err, unsigned long long timeout_ns, void* stream);

// T_m(x) by the three-term recurrence.
double cheb_T(int m, double x);

// cos(pi * a / h) for integers 0 <= a, h >= 1, with the argument reduced
// exactly (symmetry about pi/2 and pi) before one call to cos.
double cos_pi_ratio(int64_t a, int64_t h);

void set_error(const std::string& msg);
fct_status fail(fct_status s, const std::string& msg);

}  // namespace fct
