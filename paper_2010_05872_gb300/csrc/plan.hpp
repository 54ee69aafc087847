// Host-side plan of the multilevel transform: grid hierarchy, per-level
// per-axis 1D operator tables and level tolerances, all in FP64.
//
// The tables are the data the GPU kernels need for one level transition
// l -> l-1 along one axis (Section 2; Section 5.2 Lemma 1; Section 5.4):
//   iwl/iwr : linear-interpolation weights of each coefficient node from its
//             two coarse neighbours (0 on nodal nodes),
//   rw      : the load-vector (mass multiply + restriction, P^T M_f) row of
//             each coarse node, as 5 weights on fine offsets -2..+2 around the
//             coarse node's fine position,
//   ta/tm/tc: Thomas factors of the coarse mass matrix M_c: sub-diagonal a_k,
//             reciprocal pivot m_k and eliminated super-diagonal c'_k
//             (precomputed once, Section 5.4 "intermediate variable reuse").
// rw and M_c are both divided by the mean coarse spacing, which cancels in
// M_c^{-1} P^T M_f and keeps FP32 tables O(1).
#pragma once

#include <array>
#include <cstdint>
#include <vector>

namespace mgb {

constexpr int kMaxLevels = 40;

struct AxisTables {
  int n = 1;   // fine nodes on this axis at level l (1 = padded axis)
  int nc = 1;  // coarse nodes, n / 2 + 1
  std::vector<double> iwl, iwr;    // [n]
  std::vector<double> rw;          // [nc * 5]
  std::vector<double> xd, xr;      // [nc * 3] R P and R S on coarse nodes k-1, k, k+1
  std::vector<double> ta, tm, tc;  // [nc]
  // Segmented form of the two Thomas recurrences (segments of seg_len rows):
  // forward y_k = tm_k f_k + sb_k y_{k-1}, backward x_k = y_k + sy_k x_{k+1},
  // and the products sg_k (sb from the segment start to k) and sh_k (sy from
  // k to the segment end) that carry a segment's boundary value inward.
  std::vector<double> sb, sg, sy, sh;  // [nc]
  int seg_len = 1;
  double rmax = 1, smax = 1, dmax = 0;  // row-sum maxima of |M_c^{-1} P^T M_f|
};

struct HostPlan {
  int ndim = 0;                           // dimensionality given by the caller
  std::array<int64_t, 3> dims3{1, 1, 1};  // padded to 3 axes (leading 1s)
  int L = 0;
  std::vector<std::array<int64_t, 3>> shape;  // [L+1] level shapes (padded)
  std::vector<std::array<AxisTables, 3>> ax;  // [L+1]; entry l = transition l -> l-1
  std::array<std::vector<uint8_t>, 3> lev;    // per finest index: least level containing it
  std::vector<uint8_t> lev01;                 // per finest row (j0, j1): max(lev[0][j0], lev[1][j1])
  std::vector<double> knorm;                  // [L+1] bound on |K_l|_inf (entry 0 unused)
  std::vector<double> coords_key;             // coordinates as given (for the plan cache)
  std::array<std::vector<double>, 3> x;       // finest coordinates per axis (padded: {0})
  std::vector<std::array<std::vector<int64_t>, 3>> idx;  // [L+1] level-l node positions (finest indices)
  int64_t count() const { return dims3[0] * dims3[1] * dims3[2]; }
};

// Returns MGARD_OK or an MGARD_ERR_* code.
int check_shape(int ndim, const int64_t* dims);
int count_levels(int ndim, const int64_t* dims, int* L);
int build_host_plan(int ndim, const int64_t* dims, const double* const* coords, HostPlan& out);

double linf_constant(const HostPlan& p, int stop_level);
// The tables of one axis of a level transition from the level's coordinates
// (used directly by the 4D path).
void build_axis_tables(const std::vector<double>& x, AxisTables& t);

// Free the cached 4D plans of one device (the 4D grids keep their own cache).
void release_plans4(int device);

// tau_out receives L+1 values (entries below stop_level repeat tau_{stop}).
void level_tolerances(const HostPlan& p, int stop_level, double tau, double* tau_out);
// The terms of level_tolerances: C_Linf, kappa = 2^(d/2) and
// kappa^(L + 1 - stop_level); tau_l = (1 - kappa) tau / ((1 - kpow) C) x
// kappa^(l - stop_level) for l above the stopping level.
void level_tolerance_terms(const HostPlan& p, int stop_level, double* C, double* kappa,
                           double* kpow);

// mode 0: the geometric rule above; 1: L-inf-optimal widths (tau_l
// proportional to the level's new nodes, sum tau / C_Linf); 2: tau is an L2
// bound, tau_l = tau / sqrt(h_l^d #N_L) (Section 4.1).
void level_tolerances_mode(const HostPlan& p, int stop_level, double tau, int mode, double* tau_out);

}  // namespace mgb
