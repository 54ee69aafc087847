// Host plan construction: hierarchy, 1D operator tables, L-infinity constant
// and level tolerances.  See plan.hpp for what each table holds.
#include "plan.hpp"

#include <algorithm>
#include <cmath>

#include "mgard_gb.h"

namespace mgb {

namespace {

// Coarse node k of an axis with n fine nodes sits at fine position
// min(2k, n-1): every even node is kept, and for even n the last node too
// (the hierarchy rule of the header).
inline int cpos(int k, int n) { return std::min(2 * k, n - 1); }
inline bool is_coef(int j, int n) { return (j & 1) && j != n - 1; }

// One axis of a level transition, built from the level-l coordinates x.
void build_axis(const std::vector<double>& x, AxisTables& t) {
  const int n = static_cast<int>(x.size());
  const int nc = n / 2 + 1;
  t.n = n;
  t.nc = nc;
  t.iwl.assign(n, 0.0);
  t.iwr.assign(n, 0.0);
  for (int j = 1; j < n - 1; ++j) {
    if (!is_coef(j, n)) continue;
    const double span = x[j + 1] - x[j - 1];
    t.iwl[j] = (x[j + 1] - x[j]) / span;  // weight of the left coarse neighbour
    t.iwr[j] = (x[j] - x[j - 1]) / span;  // weight of the right coarse neighbour
  }
  const double hbar = (x[n - 1] - x[0]) / (nc - 1);

  // Fine P1 mass matrix entries (integrals of hat-function products):
  // diagonal (D_{i-1} + D_i)/3, neighbours D/6.
  auto mf = [&](int i, int j) -> double {
    if (j < 0 || j >= n) return 0.0;
    if (i == j) {
      double d = 0.0;
      if (i > 0) d += x[i] - x[i - 1];
      if (i < n - 1) d += x[i + 1] - x[i];
      return d / 3.0;
    }
    if (j == i + 1) return (x[i + 1] - x[i]) / 6.0;
    if (j == i - 1) return (x[i] - x[i - 1]) / 6.0;
    return 0.0;
  };
  // Load-vector row of coarse node k: R[k, j] = sum_i P[i, k] M_f[i, j] with
  // P[c, k] = 1 at the node itself and the interpolation weights of its
  // coefficient neighbours (Lemma 1 of Section 5.2 is the uniform case).
  t.rw.assign(static_cast<size_t>(nc) * 5, 0.0);
  for (int k = 0; k < nc; ++k) {
    const int c = cpos(k, n);
    int ii[3];
    double pw[3];
    int m = 0;
    ii[m] = c; pw[m++] = 1.0;
    if (c - 1 >= 0 && is_coef(c - 1, n)) { ii[m] = c - 1; pw[m++] = t.iwr[c - 1]; }
    if (c + 1 < n && is_coef(c + 1, n)) { ii[m] = c + 1; pw[m++] = t.iwl[c + 1]; }
    for (int q = 0; q < m; ++q)
      for (int j = ii[q] - 1; j <= ii[q] + 1; ++j) {
        const int off = j - c + 2;
        if (j < 0 || j >= n) continue;
        t.rw[static_cast<size_t>(k) * 5 + off] += pw[q] * mf(ii[q], j) / hbar;
      }
  }

  // The load-vector rows taken against coarse nodes, tridiagonal on the
  // coarse grid: xd = R P (P the prolongation: 1 on the node itself and the
  // interpolation weights on its coefficient neighbours; the coarse mass
  // matrix in the scaling of R) and xr = R S (S: the coarse node's own fine
  // node only).  Entry 3k + d belongs to coarse node k - 1 + d.
  t.xd.assign(static_cast<size_t>(nc) * 3, 0.0);
  t.xr.assign(static_cast<size_t>(nc) * 3, 0.0);
  for (int k = 0; k < nc; ++k) {
    const int c = cpos(k, n);
    for (int d = 0; d < 3; ++d) {
      const int kk = k - 1 + d;
      if (kk < 0 || kk >= nc) continue;
      const int ck = cpos(kk, n);
      double sd = 0.0, sr = 0.0;
      for (int off = 0; off < 5; ++off) {
        const int j = c + off - 2;
        if (j < 0 || j >= n) continue;
        double pj = 0.0;  // P[j, kk]
        if (j == ck) pj = 1.0;
        else if (is_coef(j, n) && j - 1 == ck) pj = t.iwl[j];
        else if (is_coef(j, n) && j + 1 == ck) pj = t.iwr[j];
        sd += t.rw[static_cast<size_t>(k) * 5 + off] * pj;
        if (j == ck) sr += t.rw[static_cast<size_t>(k) * 5 + off];
      }
      t.xd[static_cast<size_t>(k) * 3 + d] = sd;
      t.xr[static_cast<size_t>(k) * 3 + d] = sr;
    }
  }

  // Coarse mass matrix on the coarse coordinates and its Thomas factors.
  std::vector<double> xc(nc), a(nc, 0.0), b(nc, 0.0), cu(nc, 0.0);
  for (int k = 0; k < nc; ++k) xc[k] = x[cpos(k, n)];
  for (int k = 0; k < nc; ++k) {
    if (k > 0) { const double D = xc[k] - xc[k - 1]; a[k] = D / 6.0 / hbar; b[k] += D / 3.0 / hbar; }
    if (k < nc - 1) { const double D = xc[k + 1] - xc[k]; cu[k] = D / 6.0 / hbar; b[k] += D / 3.0 / hbar; }
  }
  t.ta = a;
  t.tm.assign(nc, 0.0);
  t.tc.assign(nc, 0.0);
  double cprev = 0.0;
  for (int k = 0; k < nc; ++k) {
    const double piv = b[k] - a[k] * cprev;
    t.tm[k] = 1.0 / piv;
    t.tc[k] = cu[k] / piv;
    cprev = t.tc[k];
  }

  // Segmented recurrences: segments of at most 16 rows, as even as possible.
  {
    const int nseg = (nc + 15) / 16;
    const int L = (nc + nseg - 1) / nseg;
    t.seg_len = L;
    t.sb.assign(nc, 0.0); t.sg.assign(nc, 0.0); t.sy.assign(nc, 0.0); t.sh.assign(nc, 0.0);
    for (int k = 0; k < nc; ++k) {
      t.sb[k] = -a[k] * t.tm[k];
      t.sy[k] = -t.tc[k];
    }
    for (int k0 = 0; k0 < nc; k0 += L) {
      const int k1 = std::min(k0 + L, nc) - 1;
      double g = 1.0;
      for (int k = k0; k <= k1; ++k) { g *= t.sb[k]; t.sg[k] = g; }
      double h = 1.0;
      for (int k = k1; k >= k0; --k) { h *= t.sy[k]; t.sh[k] = h; }
    }
  }

  // Row sums of |A| with A = M_c^{-1} P^T M_f: r over all fine columns,
  // s over the coarse (nodal) columns.  Row k of M_c^{-1} is found by a
  // Thomas solve of M_c y = e_k on a window of +-64 rows around k; the
  // entries of M_c^{-1} decay at least by half per row (M_c is diagonally
  // dominant by a factor of 2), so the window is exact to FP64 rounding.
  const int W = 64;
  std::vector<double> y, cp, dp, row;
  t.rmax = 0.0; t.smax = 0.0; t.dmax = 0.0;
  for (int k = 0; k < nc; ++k) {
    const int lo = std::max(0, k - W), hi = std::min(nc - 1, k + W);
    const int m = hi - lo + 1;
    y.assign(m, 0.0); cp.assign(m, 0.0); dp.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
      const int g = lo + i;
      const double ai = i > 0 ? a[g] : 0.0;
      const double ci = i < m - 1 ? cu[g] : 0.0;
      const double rhs = (g == k) ? 1.0 : 0.0;
      const double piv = b[g] - ai * (i > 0 ? cp[i - 1] : 0.0);
      cp[i] = ci / piv;
      dp[i] = (rhs - ai * (i > 0 ? dp[i - 1] : 0.0)) / piv;
    }
    for (int i = m - 1; i >= 0; --i) y[i] = dp[i] - (i < m - 1 ? cp[i] * y[i + 1] : 0.0);
    const int j0 = std::max(0, cpos(lo, n) - 2), j1 = std::min(n - 1, cpos(hi, n) + 2);
    row.assign(j1 - j0 + 1, 0.0);
    for (int i = 0; i < m; ++i) {
      const int g = lo + i, c = cpos(g, n);
      for (int off = 0; off < 5; ++off) {
        const int j = c + off - 2;
        if (j < 0 || j >= n) continue;
        row[j - j0] += y[i] * t.rw[static_cast<size_t>(g) * 5 + off];
      }
    }
    double r = 0.0, s = 0.0;
    for (int j = j0; j <= j1; ++j) {
      const double v = std::fabs(row[j - j0]);
      r += v;
      if (!is_coef(j, n)) s += v;
    }
    t.rmax = std::max(t.rmax, r);
    t.smax = std::max(t.smax, s);
    t.dmax = std::max(t.dmax, r - s);
  }
}

void padded_axis(AxisTables& t) {
  t.n = 1; t.nc = 1;
  t.iwl.assign(1, 0.0); t.iwr.assign(1, 0.0);
  t.rw = {0.0, 0.0, 1.0, 0.0, 0.0};
  t.xd = {0.0, 1.0, 0.0};
  t.xr = {0.0, 1.0, 0.0};
  t.ta.assign(1, 0.0); t.tm.assign(1, 1.0); t.tc.assign(1, 0.0);
  t.sb.assign(1, 0.0); t.sg.assign(1, 0.0); t.sy.assign(1, 0.0); t.sh.assign(1, 0.0);
  t.seg_len = 1;
  t.rmax = 1.0; t.smax = 1.0; t.dmax = 0.0;
}

}  // namespace

int check_shape(int ndim, const int64_t* dims) {
  if (dims == nullptr) return MGARD_ERR_ARG;
  if (ndim < 1 || ndim > 3) return MGARD_ERR_SHAPE;
  // The contiguous axis may be long; the others index CUDA grid dimensions.
  for (int d = 0; d < ndim; ++d) {
    const int64_t cap = (d == ndim - 1) ? (int64_t(1) << 30) : (int64_t(1) << 18);
    if (dims[d] < 3 || dims[d] > cap) return MGARD_ERR_SHAPE;
  }
  return MGARD_OK;
}

int count_levels(int ndim, const int64_t* dims, int* L) {
  const int rc = check_shape(ndim, dims);
  if (rc != MGARD_OK) return rc;
  int64_t cur[3];
  for (int d = 0; d < ndim; ++d) cur[d] = dims[d];
  int l = 0;
  for (;;) {
    int64_t mn = cur[0];
    for (int d = 1; d < ndim; ++d) mn = std::min(mn, cur[d]);
    if (mn <= 3) break;
    for (int d = 0; d < ndim; ++d) cur[d] = cur[d] / 2 + 1;
    ++l;
  }
  *L = l;
  return MGARD_OK;
}

int build_host_plan(int ndim, const int64_t* dims, const double* const* coords, HostPlan& p) {
  int L = 0;
  int rc = count_levels(ndim, dims, &L);
  if (rc != MGARD_OK) return rc;
  if (L + 1 > kMaxLevels) return MGARD_ERR_SHAPE;
  p = HostPlan();
  p.ndim = ndim;
  p.L = L;
  const int pad = 3 - ndim;
  for (int d = 0; d < ndim; ++d) p.dims3[pad + d] = dims[d];

  // Finest coordinates (default: node index) and their validity.
  std::array<std::vector<double>, 3> x;
  for (int d = 0; d < ndim; ++d) {
    const int64_t n = dims[d];
    x[pad + d].resize(n);
    const double* c = (coords != nullptr) ? coords[d] : nullptr;
    for (int64_t j = 0; j < n; ++j) x[pad + d][j] = c ? c[j] : static_cast<double>(j);
    for (int64_t j = 0; j < n; ++j)
      if (!std::isfinite(x[pad + d][j])) return MGARD_ERR_COORDS;
    for (int64_t j = 1; j < n; ++j)
      if (!(x[pad + d][j] > x[pad + d][j - 1])) return MGARD_ERR_COORDS;
    if (c) p.coords_key.insert(p.coords_key.end(), c, c + n);
    p.coords_key.push_back(c ? 1.0 : 0.0);
  }

  // Index maps: level-l node positions (finest indices) per axis.
  std::vector<std::array<std::vector<int64_t>, 3>> idx(L + 1);
  for (int a = 0; a < 3; ++a) {
    idx[L][a].resize(p.dims3[a]);
    for (int64_t j = 0; j < p.dims3[a]; ++j) idx[L][a][j] = j;
  }
  for (int l = L; l >= 1; --l)
    for (int a = 0; a < 3; ++a) {
      const auto& f = idx[l][a];
      auto& c = idx[l - 1][a];
      c.clear();
      if (a < pad) { c = f; continue; }
      const int n = static_cast<int>(f.size());
      for (int k = 0; k < n / 2 + 1; ++k) c.push_back(f[cpos(k, n)]);
    }
  p.shape.resize(L + 1);
  for (int l = 0; l <= L; ++l)
    for (int a = 0; a < 3; ++a) p.shape[l][a] = static_cast<int64_t>(idx[l][a].size());

  p.ax.resize(L + 1);
  p.knorm.assign(L + 1, 0.0);
  for (int l = 1; l <= L; ++l) {
    for (int a = 0; a < 3; ++a) {
      if (a < pad) { padded_axis(p.ax[l][a]); continue; }
      std::vector<double> xl(idx[l][a].size());
      for (size_t j = 0; j < xl.size(); ++j) xl[j] = x[a][idx[l][a][j]];
      build_axis(xl, p.ax[l][a]);
    }
    // Telescoping bound of max_k (prod_d r_d - prod_d s_d) over the user's
    // axes in order: sum_d (prod_{e<d} smax_e) dmax_d (prod_{e>d} rmax_e).
    double norm = 0.0;
    for (int d = 0; d < ndim; ++d) {
      double term = p.ax[l][pad + d].dmax;
      for (int e = 0; e < d; ++e) term *= p.ax[l][pad + e].smax;
      for (int e = d + 1; e < ndim; ++e) term *= p.ax[l][pad + e].rmax;
      norm += term;
    }
    p.knorm[l] = norm;
  }

  for (int a = 0; a < 3; ++a) {
    p.lev[a].assign(p.dims3[a], 0);
    if (a < pad) continue;
    std::vector<uint8_t>& lv = p.lev[a];
    std::fill(lv.begin(), lv.end(), static_cast<uint8_t>(L));
    for (int l = L - 1; l >= 0; --l)
      for (int64_t j : idx[l][a]) lv[j] = static_cast<uint8_t>(l);
  }
  p.lev01.resize(static_cast<size_t>(p.dims3[0] * p.dims3[1]));
  for (int64_t j0 = 0; j0 < p.dims3[0]; ++j0)
    for (int64_t j1 = 0; j1 < p.dims3[1]; ++j1)
      p.lev01[j0 * p.dims3[1] + j1] = std::max(p.lev[0][j0], p.lev[1][j1]);
  for (int a = 0; a < 3; ++a) p.x[a] = a < pad ? std::vector<double>{0.0} : x[a];
  p.idx = std::move(idx);
  return MGARD_OK;
}

void build_axis_tables(const std::vector<double>& x, AxisTables& t) { build_axis(x, t); }

double linf_constant(const HostPlan& p, int stop_level) {
  double C = 1.0;
  for (int l = stop_level + 1; l <= p.L; ++l) C = std::max(C, 1.0 + p.knorm[l]);
  return C;
}

void level_tolerances_mode(const HostPlan& p, int stop_level, double tau, int mode,
                           double* out) {
  if (mode == 0) {
    level_tolerances(p, stop_level, tau, out);
    return;
  }
  const int pad = 3 - p.ndim;
  auto nodes = [&](int l) { return double(p.shape[l][0]) * p.shape[l][1] * p.shape[l][2]; };
  const double nL = nodes(p.L);
  if (mode == 1) {
    // L-inf-optimal widths: tau_l proportional to #N*_l (the coarse block
    // counted whole at the stopping level), summing to tau / C_Linf.
    const double C = linf_constant(p, stop_level);
    for (int l = stop_level; l <= p.L; ++l) {
      const double cnt = l == stop_level ? nodes(l) : nodes(l) - nodes(l - 1);
      out[l] = tau / C * cnt / nL;
    }
  } else {
    // L2 control: tau_l = tau / sqrt(h_l^d #N_L), h_l^d the product of the
    // largest 1D mass-matrix row sums (integrals of the hat functions) of
    // level l.
    for (int l = stop_level; l <= p.L; ++l) {
      double hd = 1.0;
      for (int d = 0; d < p.ndim; ++d) {
        const auto& ix = p.idx[l][pad + d];
        const auto& x = p.x[pad + d];
        const size_t n = ix.size();
        double m = 0.0;
        for (size_t j = 0; j < n; ++j) {
          const double left = j > 0 ? x[ix[j]] - x[ix[j - 1]] : 0.0;
          const double right = j + 1 < n ? x[ix[j + 1]] - x[ix[j]] : 0.0;
          m = std::max(m, 0.5 * (left + right));
        }
        hd *= m;
      }
      out[l] = tau / std::sqrt(hd * nL);
    }
  }
  for (int l = 0; l < stop_level; ++l) out[l] = out[stop_level];
}

void level_tolerance_terms(const HostPlan& p, int stop_level, double* C, double* kappa,
                           double* kpow) {
  *C = linf_constant(p, stop_level);
  *kappa = std::sqrt(std::pow(2.0, p.ndim));
  double kp = 1.0;
  for (int i = 0; i < p.L + 1 - stop_level; ++i) kp *= *kappa;
  *kpow = kp;
}

void level_tolerances(const HostPlan& p, int stop_level, double tau, double* out) {
  double C, kappa, kpow;
  level_tolerance_terms(p, stop_level, &C, &kappa, &kpow);
  const double t0 = (1.0 - kappa) * tau / ((1.0 - kpow) * C);
  for (int l = 0; l <= stop_level; ++l) out[l] = t0;
  for (int l = stop_level + 1; l <= p.L; ++l) out[l] = kappa * out[l - 1];
}

}  // namespace mgb
