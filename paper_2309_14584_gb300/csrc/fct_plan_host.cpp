// Host-side plan construction for the GB300 sparse FCT: alias (fold) tables,
// bin-sorted CSR, DCT-I matrices and DCT pass work units.  Pure C++: the same
// code backs fct_plan_create and the device-free fct_alias_tables_host.
//
// Alias structure (Sec. 3.1-3.3 of the paper, Eq. (aliasing_matrix_nd_diff)
// and Eq. (L-grid_A_mat)), read on Chebyshev extrema grids with a DCT-I:
// column m of grid l's block has exactly one nonzero, in the row-major bin
//   bin_l(m) = sum_{i: n_i >= 2} fold_{n_i}(m_i) * stride_i,
//   fold_n(m) = r if r <= n-1 else 2(n-1) - r,  r = m mod 2(n-1),
// with value prod_{i: n_i = 1} T_{m_i}(xi_{l,i}).  Empty bins are dropped;
// nonempty bins of grid l become rows row_off[l] .. row_off[l+1]-1 in
// ascending bin order.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <string>

#include "fct_internal.h"

namespace fct {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

fct_status fail(fct_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

double cheb_T(int m, double x) {
  if (m == 0) return 1.0;
  double t0 = 1.0, t1 = x;
  for (int k = 1; k < m; ++k) {
    double t2 = 2.0 * x * t1 - t0;
    t0 = t1;
    t1 = t2;
  }
  return t1;
}

double cos_pi_ratio(int64_t a, int64_t h) {
  // cos(pi a / h): reduce a to [0, 2h), then to [0, h] by cos(2pi - t) = cos t,
  // then to [0, h/2] by cos(pi - t) = -cos t.
  int64_t p = 2 * h;
  a %= p;
  if (a < 0) a += p;
  if (a > h) a = p - a;
  double sign = 1.0;
  if (2 * a > h) {
    a = h - a;
    sign = -1.0;
  }
  if (2 * a == h) return 0.0;
  if (a == 0) return sign;
  return sign * std::cos(M_PI * static_cast<double>(a) / static_cast<double>(h));
}

static inline int64_t fold_index(int64_t m, int64_t n) {
  const int64_t period = 2 * (n - 1);
  const int64_t r = m % period;
  return r <= n - 1 ? r : period - r;
}

// First-kind grid of n points (the aliasing lemma): with q = m div 2n and
// r = m mod 2n, T_m's one entry in the n-row block is
//   r < n: row r, (-1)^q (1 at r = 0, else 1/2);  r > n: row 2n - r, -(-1)^q / 2;
//   r = n: none (T_m vanishes on every node) -- kept as row 0 with value 0.
static inline int64_t fold_first_kind(int64_t m, int64_t n, double* val) {
  const int64_t q = m / (2 * n), r = m % (2 * n);
  const double sgn = (q & 1) ? -1.0 : 1.0;
  if (r < n) {
    *val = r == 0 ? sgn : 0.5 * sgn;
    return r;
  }
  if (r > n) {
    *val = -0.5 * sgn;
    return 2 * n - r;
  }
  *val = 0.0;
  return 0;
}

fct_status build_host_tables(int D, int64_t N, const uint16_t* support, int K,
                             const int32_t* sizes, const double* nodes, int grid_kind, bool with_dct,
                             HostTables* out, std::string* err, bool with_alias) {
  auto bad = [&](const std::string& m) {
    *err = m;
    return FCT_ERR_INVALID_ARG;
  };
  if (D < 1 || D > kMaxD) return bad("D must be in [1, 255]");
  if (N < 1) return bad("N must be >= 1");
  if (K < 1) return bad("K must be >= 1");
  if (!support || !sizes) return bad("support and sizes must not be NULL");
  if (grid_kind != FCT_GRID_EXTREMA && grid_kind != FCT_GRID_FIRST_KIND) return bad("unknown grid kind");
  const bool first = grid_kind == FCT_GRID_FIRST_KIND;
  if (static_cast<int64_t>(K) * N >= (int64_t(1) << 31)) return bad("K*N must be below 2^31");

  HostTables& H = *out;
  H = HostTables();
  H.D = D;
  H.K = K;
  H.N = N;
  H.offsets.assign(K + 1, 0);
  for (int l = 0; l < K; ++l) {
    int64_t T = 1;
    for (int i = 0; i < D; ++i) {
      const int32_t n = sizes[l * D + i];
      if (n < 1) return bad("grid " + std::to_string(l) + " axis " + std::to_string(i) + ": size < 1");
      if (n > kMaxAxis)
        return bad("grid " + std::to_string(l) + " axis " + std::to_string(i) + ": more than " +
                   std::to_string(kMaxAxis) + " points (the direct DCT-I holds an n x n matrix per axis length)");
      T *= n;
      if (T >= (int64_t(1) << 31)) return bad("grid " + std::to_string(l) + " has 2^31 or more points");
      if (n == 1 && nodes) {
        const double xi = nodes[l * D + i];
        if (!(xi >= -1.0 && xi <= 1.0)) return bad("single-point node outside [-1, 1]");
      }
    }
    H.offsets[l + 1] = H.offsets[l] + T;
    if (H.offsets[l + 1] >= (int64_t(1) << 31)) return bad("total sample count M must be below 2^31");
  }
  H.M = H.offsets[K];

  const int64_t KN = static_cast<int64_t>(K) * N;
  if (with_alias) {
    H.bin.resize(KN);
    H.crow.resize(KN);
    H.weight.resize(KN);
    H.col.resize(KN);
    H.wcsr.resize(KN);
    H.row_off.assign(K + 1, 0);
    H.rowptr.clear();
    H.rowsrc.clear();
    H.rowgrid.clear();
    H.rowptr.push_back(0);

    // Nonzero components of every multi-index (axis order): a zero component
    // folds to bin index 0 with entry 1 on every axis kind, so only nonzero
    // components change a bin or an entry (sparse supports in high D have few).
    std::vector<int64_t> nz_off(N + 1, 0);
    std::vector<int32_t> nz_axis;
    for (int64_t m = 0; m < N; ++m) {
      for (int i = 0; i < D; ++i)
        if (support[m * D + i] != 0) nz_axis.push_back(i);
      nz_off[m + 1] = static_cast<int64_t>(nz_axis.size());
    }
    std::vector<int64_t> stride(D);
    std::vector<int32_t> count;
    std::vector<int32_t> comp;
    for (int l = 0; l < K; ++l) {
      const int32_t* sz = sizes + static_cast<int64_t>(l) * D;
      stride[D - 1] = 1;
      for (int i = D - 2; i >= 0; --i) stride[i] = stride[i + 1] * sz[i + 1];
      const int64_t T = H.offsets[l + 1] - H.offsets[l];
      int32_t* bl = H.bin.data() + static_cast<int64_t>(l) * N;
      double* wl = H.weight.data() + static_cast<int64_t>(l) * N;
      for (int64_t m = 0; m < N; ++m) {
        const uint16_t* mi = support + m * D;
        int64_t bidx = 0;
        double w = 1.0;
        for (int64_t e = nz_off[m]; e < nz_off[m + 1]; ++e) {
          const int i = nz_axis[e];
          const int32_t n = sz[i];
          if (n >= 2 && first) {
            double v = 0.0;
            bidx += fold_first_kind(mi[i], n, &v) * stride[i];
            w *= v;
          } else if (n >= 2) {
            bidx += fold_index(mi[i], n) * stride[i];
          } else {
            const double xi = nodes ? nodes[l * D + i] : 1.0;
            w *= cheb_T(mi[i], xi);
          }
        }
        bl[m] = static_cast<int32_t>(bidx);
        wl[m] = w;
      }
      // counting sort by bin (stable in m): nonempty bins in ascending order
      count.assign(static_cast<size_t>(T) + 1, 0);
      for (int64_t m = 0; m < N; ++m) count[bl[m] + 1]++;
      comp.assign(static_cast<size_t>(T), -1);
      const int32_t row0 = static_cast<int32_t>(H.rowsrc.size());
      int32_t nrows = 0;
      for (int64_t t = 0; t < T; ++t) {
        if (count[t + 1] > 0) {
          comp[t] = row0 + nrows++;
          H.rowsrc.push_back(static_cast<int32_t>(H.offsets[l] + t));
          H.rowgrid.push_back(l);
          H.rowptr.push_back(H.rowptr.back() + count[t + 1]);
        }
      }
      // scatter columns into CSR, m ascending within each bin
      std::vector<int32_t> fill(nrows, 0);
      for (int64_t m = 0; m < N; ++m) {
        const int32_t r = comp[bl[m]];
        H.crow[static_cast<int64_t>(l) * N + m] = r;
        const int32_t pos = H.rowptr[r] + fill[r - row0]++;
        H.col[pos] = static_cast<int32_t>(m);
        H.wcsr[pos] = wl[m];
      }
      H.row_off[l + 1] = row0 + nrows;
    }
    H.R = static_cast<int64_t>(H.rowsrc.size());
  }  // with_alias

  // node positions of every grid axis (used by the sampler)
  H.node_off.resize(static_cast<size_t>(K) * D);
  H.node_pos.clear();
  for (int l = 0; l < K; ++l) {
    for (int i = 0; i < D; ++i) {
      const int32_t n = sizes[l * D + i];
      H.node_off[l * D + i] = static_cast<int32_t>(H.node_pos.size());
      if (n == 1) {
        H.node_pos.push_back(nodes ? nodes[l * D + i] : 1.0);
      } else if (first) {
        for (int j = 0; j < n; ++j) H.node_pos.push_back(cos_pi_ratio(2 * j + 1, 2 * static_cast<int64_t>(n)));
      } else {
        for (int j = 0; j < n; ++j) H.node_pos.push_back(cos_pi_ratio(j, n - 1));
      }
    }
  }

  if (!with_dct) return FCT_OK;

  // DCT matrices, one per distinct axis length.  Extrema grid, the DCT-I
  // interpolation: C[k][j] = (2 e_k/(n-1)) e_j cos(pi (j k mod 2(n-1))/(n-1)),
  // e = 1/2 at the ends.  First-kind grid, the quadrature of the aliasing
  // lemma: C[k][j] = cos(pi (k (2j + 1) mod 4n) / 2n) / n.
  std::vector<int32_t> mat_of(1, -1);
  auto matrix_for = [&](int32_t n) -> int32_t {
    if (static_cast<int32_t>(mat_of.size()) <= n) mat_of.resize(n + 1, -1);
    if (mat_of[n] >= 0) return mat_of[n];
    const int32_t off = static_cast<int32_t>(H.dct_mats.size());
    if (n == 1) {
      H.dct_mats.push_back(1.0);
    } else if (first) {
      const int64_t h = 2 * static_cast<int64_t>(n);
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          H.dct_mats.push_back(cos_pi_ratio((static_cast<int64_t>(k) * (2 * j + 1)) % (2 * h), h) /
                               static_cast<double>(n));
    } else {
      const int64_t h = n - 1;
      for (int k = 0; k < n; ++k) {
        const double ek = (k == 0 || k == n - 1) ? 0.5 : 1.0;
        for (int j = 0; j < n; ++j) {
          const double ej = (j == 0 || j == n - 1) ? 0.5 : 1.0;
          H.dct_mats.push_back((2.0 * ek / static_cast<double>(h)) * ej *
                               cos_pi_ratio((static_cast<int64_t>(j) * k) % (2 * h), h));
        }
      }
    }
    mat_of[n] = off;
    return off;
  };

  // Active axes of every grid, outermost first.  Every axis but the last is a
  // full pass over the grid (ping-pong y0 / y1); the last is evaluated only at
  // the nonempty bins, fused with the gather of b.  A grid with no active axis
  // gets an identity "axis" (n = 1) as its last pass.
  std::vector<std::vector<int>> active(K);
  int npass = 0;
  H.gfinal.assign(K, GridFinal{});
  for (int l = 0; l < K; ++l) {
    for (int i = 0; i < D; ++i)
      if (sizes[l * D + i] >= 2) active[l].push_back(i);
    const int A = static_cast<int>(active[l].size());
    npass = std::max(npass, A - 1);
    GridFinal g{};
    if (A == 0) {
      g.n = 1;
      g.stride = 1;
      g.mat = matrix_for(1);
      g.in_sel = 0;
    } else {
      const int axis = active[l][A - 1];
      g.n = sizes[l * D + axis];
      int64_t st = 1;
      for (int i = axis + 1; i < D; ++i) st *= sizes[l * D + i];
      g.stride = static_cast<int32_t>(st);
      g.mat = matrix_for(g.n);
      g.in_sel = A == 1 ? 0 : (((A - 2) & 1) ? 2 : 1);
    }
    H.gfinal[l] = g;
  }
  // Evaluation passes of the sampler: every active axis, E[j][k] = T_k(x_j)
  // (first-kind grid: times 2 for k > 0, since its bins hold T_k's
  // coefficient halved),
  // pass p reads y0 (p = 0) or the previous output and the last pass writes
  // the caller's samples; a grid without active axes gets one copy pass.
  {
    std::vector<int32_t> emat_of;
    auto eval_for = [&](int32_t n) -> int32_t {
      if (static_cast<int32_t>(emat_of.size()) <= n) emat_of.resize(n + 1, -1);
      if (emat_of[n] >= 0) return emat_of[n];
      const int32_t off = static_cast<int32_t>(H.eval_mats.size());
      if (n == 1) {
        H.eval_mats.push_back(1.0);
      } else if (first) {
        const int64_t h = 2 * static_cast<int64_t>(n);
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k)
            H.eval_mats.push_back((k == 0 ? 1.0 : 2.0) *
                                  cos_pi_ratio((static_cast<int64_t>(k) * (2 * j + 1)) % (2 * h), h));
      } else {
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k)
            H.eval_mats.push_back(cos_pi_ratio((static_cast<int64_t>(j) * k) % (2 * (n - 1)), n - 1));
      }
      emat_of[n] = off;
      return off;
    };
    int nip = 0;
    for (int l = 0; l < K; ++l) nip = std::max<int>(nip, std::max<size_t>(1, active[l].size()));
    H.nipass = nip;
    H.ipass_chunk_off.assign(1, 0);
    for (int p = 0; p < nip; ++p) {
      for (int l = 0; l < K; ++l) {
        const int A = std::max<int>(1, static_cast<int>(active[l].size()));
        if (p >= A) continue;
        int32_t n = 1;
        int64_t st = 1;
        if (!active[l].empty()) {
          const int axis = active[l][p];
          n = sizes[l * D + axis];
          for (int i = axis + 1; i < D; ++i) st *= sizes[l * D + i];
        }
        const int32_t mat = eval_for(n);
        const int8_t in_sel = p == 0 ? 1 : static_cast<int8_t>(((p - 1) & 1) ? 1 : 2);
        const int8_t out_sel = p == A - 1 ? 3 : static_cast<int8_t>((p & 1) ? 1 : 2);
        const int64_t T = H.offsets[l + 1] - H.offsets[l];
        for (int64_t e0 = 0; e0 < T; e0 += kDctChunk) {
          DctChunk c{};
          c.base = H.offsets[l];
          c.start = static_cast<int32_t>(e0);
          c.count = static_cast<int32_t>(std::min<int64_t>(kDctChunk, T - e0));
          c.n = n;
          c.stride = static_cast<int32_t>(st);
          c.mat = mat;
          c.in_sel = in_sel;
          c.out_sel = out_sel;
          H.idct_chunks.push_back(c);
        }
      }
      H.ipass_chunk_off.push_back(static_cast<int32_t>(H.idct_chunks.size()));
    }
  }

  H.npass = npass;
  H.pass_chunk_off.assign(1, 0);
  for (int p = 0; p < npass; ++p) {
    // fibres of this pass over all grids: one thread per fibre pays only when
    // they fill the GPU several times over (else one thread per output)
    int64_t pass_fibres = 0;
    for (int l = 0; l < K; ++l) {
      const int A = static_cast<int>(active[l].size());
      if (p >= A - 1) continue;
      pass_fibres += (H.offsets[l + 1] - H.offsets[l]) / sizes[l * D + active[l][p]];
    }
    for (int l = 0; l < K; ++l) {
      const int A = static_cast<int>(active[l].size());
      if (p >= A - 1) continue;
      const int axis = active[l][p];
      const int32_t n = sizes[l * D + axis];
      int64_t st = 1;
      for (int i = axis + 1; i < D; ++i) st *= sizes[l * D + i];
      const int32_t mat = matrix_for(n);
      const int8_t out_sel = static_cast<int8_t>((p & 1) ? 2 : 1);
      const int8_t in_sel = p == 0 ? 0 : static_cast<int8_t>(((p - 1) & 1) ? 2 : 1);
      const int64_t T = H.offsets[l + 1] - H.offsets[l];
      // short axes: units of fibres (one thread computes a fibre's n outputs);
      // longer ones: units of output elements (one thread per output)
      const bool by_fibre = n >= kFibreMinN && n <= kFibreMaxN && pass_fibres >= kFibrePassMin;
      const int64_t units = by_fibre ? T / n : T;
      const int64_t per = by_fibre ? kFibreChunk : kDctChunk;
      for (int64_t e0 = 0; e0 < units; e0 += per) {
        DctChunk c{};
        c.base = H.offsets[l];
        c.start = static_cast<int32_t>(e0);
        c.count = static_cast<int32_t>(std::min<int64_t>(per, units - e0));
        c.n = n;
        c.stride = static_cast<int32_t>(st);
        c.mat = mat;
        c.in_sel = in_sel;
        c.out_sel = out_sel;
        c.fibres = by_fibre ? 1 : 0;
        H.dct_chunks.push_back(c);
      }
    }
    H.pass_chunk_off.push_back(static_cast<int32_t>(H.dct_chunks.size()));
  }
  return FCT_OK;
}

void device_row_order(HostTables* Hp, int epl) {
  HostTables& H = *Hp;
  const int64_t R = H.R;
  std::vector<int32_t> order(R);
  for (int64_t r = 0; r < R; ++r) order[r] = static_cast<int32_t>(r);
  // stable sort by row_order_key: gather lane class, then (32-lane and wide
  // rows of large plans) load rounds, longest first; equal keys keep their
  // bin order, which keeps neighbouring coefficients' rows close together
  const bool by_rounds = static_cast<int64_t>(H.K) * H.N >= kRoundsOrderMinEntries;
  std::vector<int32_t> key(R);
  for (int64_t r = 0; r < R; ++r) {
    const int32_t len = H.rowptr[r + 1] - H.rowptr[r];
    key[r] = row_order_key(len, lanes_for(len, epl), epl, by_rounds);
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  std::vector<int32_t> inv(R), rowptr(R + 1), col(H.col.size()), rowsrc(R), rowgrid(R);
  std::vector<double> wcsr(H.wcsr.size());
  rowptr[0] = 0;
  for (int64_t nr = 0; nr < R; ++nr) {
    const int32_t r = order[nr];
    inv[r] = static_cast<int32_t>(nr);
    const int32_t len = H.rowptr[r + 1] - H.rowptr[r];
    rowptr[nr + 1] = rowptr[nr] + len;
    std::copy(H.col.begin() + H.rowptr[r], H.col.begin() + H.rowptr[r + 1], col.begin() + rowptr[nr]);
    std::copy(H.wcsr.begin() + H.rowptr[r], H.wcsr.begin() + H.rowptr[r + 1], wcsr.begin() + rowptr[nr]);
    rowsrc[nr] = H.rowsrc[r];
    rowgrid[nr] = H.rowgrid[r];
  }
  for (auto& c : H.crow) c = inv[c];
  H.rowptr.swap(rowptr);
  H.col.swap(col);
  H.wcsr.swap(wcsr);
  H.rowsrc.swap(rowsrc);
  H.rowgrid.swap(rowgrid);
}

int lanes_for(int32_t len, int epl) {
  int lanes = 1;
  while (lanes < 32 && lanes * epl < len) lanes <<= 1;
  if (len > kWideRowFactor * 32 * epl) return kWideLanes;
  return lanes;
}

// rows of one unit: workers / lanes, one for a wide row
static inline int rows_per_unit(int lanes, int workers) { return lanes > 32 ? 1 : workers / lanes; }

int64_t units_from_classes(const int64_t* per_class, int workers) {
  int64_t units = 0;
  for (int c = 0; c < kLaneClasses; ++c) {
    const int64_t per = rows_per_unit(1 << c, workers);
    units += (per_class[c] + per - 1) / per;
  }
  return units;
}

int pick_entries_per_lane(const int64_t classes[3][kLaneClasses], int workers, int64_t wave, int fixed) {
  if (fixed > 0) return fixed;
  if (wave > 0)
    for (int q = 0; q < 3; ++q)
      if (units_from_classes(classes[q], workers) <= wave) return 2 << q;
  return 8;
}

void lane_class_counts(const HostTables& H, int64_t classes[3][kLaneClasses]) {
  // rows sorted or not, the unit count only depends on the rows per lane class
  for (int q = 0; q < 3; ++q)
    for (int c = 0; c < kLaneClasses; ++c) classes[q][c] = 0;
  for (int64_t r = 0; r < H.R; ++r) {
    const int32_t len = H.rowptr[r + 1] - H.rowptr[r];
    for (int q = 0; q < 3; ++q) classes[q][__builtin_ctz(static_cast<unsigned>(lanes_for(len, 2 << q)))]++;
  }
}

void row_units(const HostTables& H, int workers, int epl, std::vector<int32_t>* first, std::vector<int32_t>* lanes) {
  first->clear();
  lanes->clear();
  int64_t r = 0;
  while (r < H.R) {
    const int lc = lanes_for(H.rowptr[r + 1] - H.rowptr[r], epl);
    const int per = rows_per_unit(lc, workers);
    int64_t e = r;
    // rows are sorted by lane class, so equal lane counts are contiguous
    while (e < H.R && e - r < per && lanes_for(H.rowptr[e + 1] - H.rowptr[e], epl) == lc) ++e;
    first->push_back(static_cast<int32_t>(r));
    lanes->push_back(lc);
    r = e;
  }
  first->push_back(static_cast<int32_t>(H.R));  // sentinel: end of the last unit
}

void final_pass_rows(const HostTables& H, std::vector<int32_t>* rowbase, std::vector<int32_t>* rowk) {
  rowbase->resize(H.R);
  rowk->resize(H.R);
  for (int64_t r = 0; r < H.R; ++r) {
    const int l = H.rowgrid[r];
    const GridFinal& g = H.gfinal[l];
    const int64_t bin = H.rowsrc[r] - H.offsets[l];
    const int64_t k = (bin / g.stride) % g.n;
    (*rowbase)[r] = static_cast<int32_t>(H.offsets[l] + bin - k * g.stride);
    (*rowk)[r] = static_cast<int32_t>(k);
  }
}

int64_t normal_matrix_bound(const HostTables& H) {
  int64_t b = 0;
  for (int64_t r = 0; r < H.R; ++r) {
    const int64_t len = H.rowptr[r + 1] - H.rowptr[r];
    b += len * len;
  }
  return b;
}

void normal_matrix(const HostTables& H, std::vector<int32_t>* rowptr, std::vector<int32_t>* col,
                   std::vector<double>* val) {
  // W[m][m'] = sum over grids l of w_l(m) * (entry of m' in the row of m on grid l);
  // the grids are visited in order and each row in CSR order, so the sums have a
  // fixed order.  Columns of a row come out ascending.
  const int64_t N = H.N;
  std::vector<double> acc(N, 0.0);
  std::vector<char> mark(N, 0);
  std::vector<int32_t> touched;
  rowptr->assign(N + 1, 0);
  col->clear();
  val->clear();
  for (int64_t m = 0; m < N; ++m) {
    touched.clear();
    for (int l = 0; l < H.K; ++l) {
      const int64_t e = static_cast<int64_t>(l) * N + m;
      const int32_t row = H.crow[e];
      const double wm = H.weight[e];
      for (int32_t j = H.rowptr[row]; j < H.rowptr[row + 1]; ++j) {
        const int32_t c = H.col[j];
        if (!mark[c]) {
          mark[c] = 1;
          touched.push_back(c);
        }
        acc[c] += wm * H.wcsr[j];
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int32_t c : touched) {
      col->push_back(c);
      val->push_back(acc[c]);
      acc[c] = 0.0;
      mark[c] = 0;
    }
    (*rowptr)[m + 1] = static_cast<int32_t>(col->size());
  }
}

void final_pass_rows_for(const HostTables& H, const std::vector<GridFinal>& gfinal, std::vector<int32_t>* rowbase,
                         std::vector<int32_t>* rowk) {
  rowbase->resize(H.R);
  rowk->resize(H.R);
  for (int64_t r = 0; r < H.R; ++r) {
    const int64_t src = H.rowsrc[r];
    const int l = static_cast<int>(std::upper_bound(H.offsets.begin(), H.offsets.end(), src) - H.offsets.begin()) - 1;
    const GridFinal& g = gfinal[l];
    const int64_t bin = src - H.offsets[l];
    const int64_t k = (bin / g.stride) % g.n;
    (*rowbase)[r] = static_cast<int32_t>(H.offsets[l] + bin - k * g.stride);
    (*rowk)[r] = static_cast<int32_t>(k);
  }
}

namespace {

// Balanced base-128 digits of round(v * 2^(56 - e)) (|v| < 2^e): the value is
// sum_t digit[t] 2^(7 (7 - t)), digit[0] in [-128, 128], the others in
// [-64, 63]; every digit is exact in BF16.
void tc_digits(double v, int e, int32_t digit[kTcSlices]) {
  int64_t x = std::llrint(std::ldexp(v, 56 - e));
  for (int t = kTcSlices - 1; t >= 1; --t) {
    const int64_t q = (x + 64) >> 7;  // floor((x + 64) / 128)
    digit[t] = static_cast<int32_t>(x - q * 128);
    x = q;
  }
  digit[0] = static_cast<int32_t>(x);
}

uint16_t bf16_bits_of_small_int(int32_t d) {
  const float f = static_cast<float>(d);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return static_cast<uint16_t>(u >> 16);  // exact: |d| <= 128 has at most 8 significant bits
}

// Byte offset of element (row r, k) inside one slice tile of `rows` x 16
// (K-major, no swizzle: 8 x 16-byte core matrices, the two K halves 128
// bytes apart, 8-row groups 256 bytes apart).
inline int64_t tc_tile_offset(int r, int k) { return (r / 8) * 256 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2; }

}  // namespace

fct_status build_tc_host(HostTables* Hp, const int32_t* sizes, int grid_kind, int mode, TcHost* T) {
  HostTables& H = *Hp;
  *T = TcHost{};
  if (mode < 0) return FCT_OK;
  const int K = H.K, D = H.D;
  const bool first = grid_kind == FCT_GRID_FIRST_KIND;
  std::vector<std::vector<int>> active(K);
  std::vector<char> tc(K, 0);
  bool any = false;
  for (int l = 0; l < K; ++l) {
    int longest = 0;
    for (int i = 0; i < D; ++i)
      if (sizes[l * D + i] >= 2) {
        active[l].push_back(i);
        longest = std::max(longest, sizes[l * D + i]);
      }
    if (!active[l].empty() && longest <= kTcMaxAxis && (mode == 1 || longest >= kTcMinAxis)) {
      tc[l] = 1;
      any = true;
    }
  }
  if (!any) return FCT_OK;
  T->grid_tc = tc;

  // A slices of the DCT matrix of every axis length the tensor-core grids use
  std::vector<int64_t> a_off_of(kTcMaxAxis + 1, -1);
  std::vector<int32_t> e_off_of(kTcMaxAxis + 1, -1);
  int64_t a_bytes = 0;
  for (int l = 0; l < K; ++l) {
    if (!tc[l]) continue;
    for (int i : active[l]) {
      const int n = sizes[l * D + i];
      if (a_off_of[n] >= 0) continue;
      const int ksteps = (n + kTcK - 1) / kTcK, mtiles = (n + kTcM - 1) / kTcM;
      a_off_of[n] = a_bytes;
      e_off_of[n] = static_cast<int32_t>(T->a_exp.size());
      a_bytes += static_cast<int64_t>(mtiles) * ksteps * kTcAStep;
      T->a_bits.resize(a_bytes / 2, 0);
      T->a_exp.resize(T->a_exp.size() + static_cast<size_t>(mtiles) * kTcM, 0);
      for (int k = 0; k < n; ++k) {
        // row k of the pass matrix, as build_host_tables forms it
        std::vector<double> row(n);
        double m = 0.0;
        for (int j = 0; j < n; ++j) {
          double c;
          if (first) {
            const int64_t h = 2 * static_cast<int64_t>(n);
            c = cos_pi_ratio((static_cast<int64_t>(k) * (2 * j + 1)) % (2 * h), h) / static_cast<double>(n);
          } else {
            const int64_t h = n - 1;
            const double ek = (k == 0 || k == n - 1) ? 0.5 : 1.0;
            const double ej = (j == 0 || j == n - 1) ? 0.5 : 1.0;
            c = (2.0 * ek / static_cast<double>(h)) * ej * cos_pi_ratio((static_cast<int64_t>(j) * k) % (2 * h), h);
          }
          row[j] = c;
          m = std::max(m, std::fabs(c));
        }
        int e = 0;
        if (m > 0.0) std::frexp(m, &e);
        T->a_exp[e_off_of[n] + k] = e;
        const int mt = k / kTcM, r = k % kTcM;
        for (int j = 0; j < n; ++j) {
          int32_t dg[kTcSlices];
          tc_digits(row[j], e, dg);
          const int ks = j / kTcK, kk = j % kTcK;
          for (int t = 0; t < kTcSlices; ++t) {
            const int64_t byte = a_off_of[n] + ((static_cast<int64_t>(mt) * ksteps + ks) * kTcSlices + t) * kTcATile +
                                 tc_tile_offset(r, kk);
            T->a_bits[byte / 2] = bf16_bits_of_small_int(dg[t]);
          }
        }
      }
    }
  }

  // passes: pass p transforms the p-th active axis of every tensor-core grid
  // (ping-pong y0 / y1 as the FP64 passes do)
  int npass = 0;
  for (int l = 0; l < K; ++l)
    if (tc[l]) npass = std::max<int>(npass, static_cast<int>(active[l].size()));
  T->npass = npass;
  T->gp_off.assign(1, 0);
  T->split_off.assign(1, 0);
  T->gemm_off.assign(1, 0);
  for (int p = 0; p < npass; ++p) {
    int64_t b_off = 0, f_off = 0;
    for (int l = 0; l < K; ++l) {
      const int A = static_cast<int>(active[l].size());
      if (!tc[l] || p >= A) continue;
      const int axis = active[l][p];
      TcGridPass g{};
      g.base = H.offsets[l];
      g.n = sizes[l * D + axis];
      int64_t post = 1;
      for (int i = axis + 1; i < D; ++i) post *= sizes[l * D + i];
      const int64_t Tl = H.offsets[l + 1] - H.offsets[l];
      g.post = static_cast<int32_t>(post);
      g.ncols = static_cast<int32_t>(Tl / g.n);
      g.ksteps = (g.n + kTcK - 1) / kTcK;
      T->max_ksteps = std::max(T->max_ksteps, g.ksteps);
      g.mtiles = (g.n + kTcM - 1) / kTcM;
      g.ntiles = (g.ncols + kTcN - 1) / kTcN;
      g.a_off = a_off_of[g.n];
      g.e_off = e_off_of[g.n];
      g.b_off = b_off;
      g.f_off = static_cast<int32_t>(f_off);
      g.in_sel = p == 0 ? 0 : static_cast<int8_t>(((p - 1) & 1) ? 2 : 1);
      g.out_sel = static_cast<int8_t>((p & 1) ? 2 : 1);
      b_off += static_cast<int64_t>(g.ntiles) * g.ksteps * kTcBStep;
      f_off += static_cast<int64_t>(g.ntiles) * kTcN;
      const int gi = static_cast<int>(T->gp.size());
      T->gp.push_back(g);
      for (int nt = 0; nt < g.ntiles; ++nt) {
        T->split_tasks.push_back(gi);
        T->split_tasks.push_back(nt);
        for (int mt = 0; mt < g.mtiles; ++mt) {
          T->gemm_tasks.push_back(gi);
          T->gemm_tasks.push_back(mt);
          T->gemm_tasks.push_back(nt);
          T->gemm_tasks.push_back(0);
        }
      }
    }
    T->b_bytes = std::max(T->b_bytes, b_off);
    T->f_count = std::max(T->f_count, f_off);
    T->gp_off.push_back(static_cast<int32_t>(T->gp.size()));
    T->split_off.push_back(static_cast<int32_t>(T->split_tasks.size() / 2));
    T->gemm_off.push_back(static_cast<int32_t>(T->gemm_tasks.size() / 4));
  }
  if (T->f_count > (int64_t{1} << 31) || T->b_bytes > (int64_t{1} << 40)) return FCT_ERR_INVALID_ARG;

  // the solver's DCT when the tensor-core passes ran first: the FP64 passes of
  // the other grids (a pass list without the tensor-core grids' units), and an
  // identity last pass that reads each tensor-core grid's finished transform
  int32_t ident = -1;
  for (const GridFinal& g : H.gfinal)
    if (g.n == 1) ident = g.mat;
  if (ident < 0) {
    ident = static_cast<int32_t>(H.dct_mats.size());
    H.dct_mats.push_back(1.0);
  }
  T->gfinal = H.gfinal;
  for (int l = 0; l < K; ++l) {
    if (!tc[l]) continue;
    const int A = static_cast<int>(active[l].size());
    GridFinal g{};
    g.n = 1;
    g.stride = 1;
    g.mat = ident;
    g.in_sel = ((A - 1) & 1) ? 2 : 1;
    T->gfinal[l] = g;
  }
  T->pass_chunk_off.assign(1, 0);
  for (int p = 0; p < H.npass; ++p) {
    for (int32_t c = H.pass_chunk_off[p]; c < H.pass_chunk_off[p + 1]; ++c) {
      const DctChunk& ch = H.dct_chunks[c];
      const int l = static_cast<int>(std::upper_bound(H.offsets.begin(), H.offsets.end(), ch.base) -
                                     H.offsets.begin()) - 1;
      if (!tc[l]) T->dct_chunks.push_back(ch);
    }
    if (static_cast<int32_t>(T->dct_chunks.size()) == T->pass_chunk_off.back()) break;
    T->pass_chunk_off.push_back(static_cast<int32_t>(T->dct_chunks.size()));
    T->npass_fp64 = p + 1;
  }
  return FCT_OK;
}

}  // namespace fct

extern "C" {

const char* fct_last_error(void) { return fct::g_last_error.c_str(); }

const char* fct_status_string(int s) {
  switch (s) {
    case FCT_OK: return "FCT_OK";
    case FCT_ERR_INVALID_ARG: return "FCT_ERR_INVALID_ARG";
    case FCT_ERR_RANK: return "FCT_ERR_RANK";
    case FCT_ERR_NOCONV: return "FCT_ERR_NOCONV";
    case FCT_ERR_TIMEOUT: return "FCT_ERR_TIMEOUT";
    case FCT_ERR_OOM: return "FCT_ERR_OOM";
    case FCT_ERR_NONFINITE: return "FCT_ERR_NONFINITE";
    case FCT_ERR_CUDA: return "FCT_ERR_CUDA";
    case FCT_ERR_NO_DEVICE: return "FCT_ERR_NO_DEVICE";
    default: return "FCT_ERR_UNKNOWN";
  }
}

void fct_default_options(fct_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = FCT_FP64;
  opt->tol = 1e-13;
  opt->max_iter = 50000;
  opt->inner_tol = 1e-6;
  opt->max_refine = 6;
  opt->block_threads = 0;
  opt->max_blocks = 0;
  opt->coef_lanes = 0;
  opt->timeout_s = 4.0;
  opt->normal_matrix = 0;
  opt->grid_kind = FCT_GRID_EXTREMA;
  opt->entries_per_lane = 0;
  opt->plan_build = FCT_PLAN_BUILD_AUTO;
}

fct_status fct_alias_tables_host(int D, int64_t N, const uint16_t* support, int K,
                                 const int32_t* sizes, const double* nodes, int grid_kind, int32_t* bin,
                                 int32_t* crow, double* weight, int64_t* R_out) {
  fct::HostTables H;
  std::string err;
  fct_status s = fct::build_host_tables(D, N, support, K, sizes, nodes, grid_kind, false, &H, &err);
  if (s != FCT_OK) return fct::fail(s, err);
  const size_t KN = static_cast<size_t>(K) * static_cast<size_t>(N);
  if (bin) std::memcpy(bin, H.bin.data(), KN * sizeof(int32_t));
  if (crow) std::memcpy(crow, H.crow.data(), KN * sizeof(int32_t));
  if (weight) std::memcpy(weight, H.weight.data(), KN * sizeof(double));
  if (R_out) *R_out = H.R;
  return FCT_OK;
}

}  // extern "C"
