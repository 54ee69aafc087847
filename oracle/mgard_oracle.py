"""FP64 CPU oracle for MGARD+ multilevel decomposition, recomposition and
level-wise quantization (Liang et al., "MGARD+: Optimizing Multilevel Methods
for Error-bounded Scientific Data Reduction", arXiv 2010.05872).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py``.  The product path (the CUDA library and its Python
binding) never imports it, and it imports nothing from the product package.

What it computes is the plain definition of the transform, written with
explicit finite-element operators assembled from the grid coordinates:

* ``Q_{l-1}`` is the L2 projection from the level-l piecewise-multilinear
  space onto the level-(l-1) one (Section 2, "Background"): per axis
  ``A_d = M_c^{-1} P^T M_f`` with ``M`` the P1 mass matrix (integrals of
  products of hat functions), ``P`` the 1D linear prolongation and
  ``M_c`` assembled from the coarse coordinates; the tensor-product operator is
  applied one axis at a time (axis d-1 first).
* ``Pi_{l-1}`` is multilinear interpolation from the coarse nodes
  (Section 2; the 1/2, 1/4, 1/8 stencils of Eq. (multilinear_interp) in
  Section 4.2 are its uniform-grid case).
* Decomposition (Section 2, decomposition steps 1-6) stores
  ``(I - Pi_{l-1}) Q_l u`` at the coefficient nodes ``N*_l`` and ``Q_{l~} u``
  on ``N_{l~}``.  Unlike the paper's route (interpolant, then the correction
  computed from the coefficients only), the oracle forms ``Q_{l-1} u``
  directly as the projection of the level-l function; the paper's identity
  ``Q_{l-1}u = u|_{N_{l-1}} + Q_{l-1}(I - Pi_{l-1})Q_l u`` is checked in the
  tests instead of being used here.
* Recomposition (Section 2, recomposition steps 1-5): the correction
  ``z = Q_{l-1}(w)`` of the coefficient function ``w``, subtraction, then
  interpolation plus coefficients.
* Level tolerances: Eq. (LinfTau) of Section 4.1 with the stopping level of
  Algorithm 1: ``tau_l~ = (1-k) tau / ((1-k^(L+1-l~)) C)``,
  ``tau_l = k tau_{l-1}``, ``k = sqrt(2^d)``.
* Quantizer (Section 4.1): zero-centred bins of width ``q_l = 2 tau_l``,
  label ``round(x / q_l)`` with ties away from zero, value ``label * q_l``.
* Adaptive stopping level (Section 4.2; the stopping-level search of
  Algorithm 1): sampled sums of the Lorenzo and interpolation prediction errors with the paper's
  penalty factors, level by level from the finest.
* Progressive recomposition (Section 1, data refactoring): ``Q_k u`` on the
  level-k grid from the decomposed array; and the iso-surface area of a 3D
  grid function (Section 6.2.2's analysis) by marching tetrahedra.
* The labels' lossless stage (the last step of Algorithm 1; this library's
  coder is a chunked zigzag bit packing, a reading) and PSNR (Section 6, "Quality").
* The other bin-width rules of Section 4.1: L-infinity-optimal widths and
  L2 error control.
* The coarse part's Lorenzo coder (the coarse part's coder in Algorithm 1):
  Lorenzo residuals of the coarse block's labels and their inverse.
* The labels' order-0 entropy and the cost model of Section 4.1, and a
  canonical Huffman coder of the labels (a reading of Algorithm 1's final
  lossless encoder, which the paper does not name).

Readings of points the paper leaves open (non-dyadic hierarchy, depth for
non-cubic shapes, the constant ``C_Linf``) are documented beside the functions
that implement them.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(exact rationals from the finite-element definition, quadrature-based
orthogonality, Lemma 1 and the printed mass matrix of Section 5.4, the
interpolation stencils of Eq. (multilinear_interp), dense Kronecker brute
force, invariants and bounds; the adaptive stopping level by hand-derived
sums in tests/golden/prediction_errors.txt and exactness properties of the
two predictors; partial recomposition by the projection chain; the iso
area by planar surfaces, exact, and a sphere's convergence; the packed
label stream by hand-derived bytes in tests/golden/packed_labels.txt and
round trips; PSNR by a closed form; the L2 and L-inf-optimal rules by a
closed form, their sums, and worst-case coefficient errors staying within
the bound after recomposition; the Lorenzo coder by hand residuals and
round trips; the entropy and cost model by closed forms and a hand count;
the Huffman coder by the textbook six-symbol example, brute-force optimal
lengths on small alphabets, Kraft's equality, the entropy bound, hand
streams in tests/golden/huffman_streams.txt and round trips).  The L2 rule's constant C_L2 = 1 is a
reading (the paper gives no value), derived and pinned as a valid bound.
``linf_constant`` is a reading (the paper
gives no value for ``C_Linf``); it is pinned only as a valid upper bound on the
worst-case error amplification, and its exact value is "parity unpinned" with
respect to the paper.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
from scipy.linalg import solve_banded

__all__ = [
    "coarse_indices", "Hierarchy", "mass_matrix", "prolongation",
    "project_axis", "project", "interpolate", "decompose", "recompose",
    "linf_constant", "level_tolerances", "node_levels", "llround",
    "quantize", "dequantize", "value_range",
    "LORENZO_PENALTY", "INTERP_PENALTY", "sampled_blocks", "prediction_errors",
    "adaptive_stop_level", "recompose_partial", "iso_area",
    "PACK_CHUNK", "pack_labels", "unpack_labels", "psnr",
    "level_tolerances_mode", "l2_error", "lorenzo_encode", "lorenzo_decode",
]


# --------------------------------------------------------------------------
# Grid hierarchy (Section 2, "Background"; Fig. 1)
# --------------------------------------------------------------------------

def coarse_indices(n: int) -> np.ndarray:
    """Indices, within one axis of ``n`` level-l nodes, of the nodes that the
    level-(l-1) grid keeps.

    Section 2 only asks for nested grids ``N_{l-1} subset N_l``; for sizes
    that are not ``2^k + 1`` the paper says MGARD+ adds dummy nodes during
    reordering (Section 6.2.2) without defining them.  Reading used here: keep
    every even index, and when ``n`` is even keep the last node too, so the
    last coarse cell has no midpoint.  The coarse size is ``n // 2 + 1``.
    """
    if n < 2:
        raise ValueError("an axis needs at least 2 nodes to coarsen")
    keep = list(range(0, n, 2))
    if n % 2 == 0:
        keep.append(n - 1)
    return np.asarray(keep, dtype=np.int64)


@dataclass
class AxisOps:
    """1D operators between level l and level l-1 along one axis."""
    keep: np.ndarray          # coarse node positions inside the fine axis
    Mf: sp.csr_matrix         # fine P1 mass matrix (n x n)
    P: sp.csr_matrix          # linear prolongation (n x n')
    Mc: sp.csr_matrix         # coarse P1 mass matrix (n' x n')


class Hierarchy:
    """Nested tensor-product grids ``N_L > ... > N_0`` (Section 2).

    ``levels[l]`` is the shape of ``N_l``; ``index[l][d]`` maps level-l node
    positions on axis ``d`` to finest-grid indices; ``coords[l][d]`` are their
    coordinates.  Every axis is coarsened at every level and the hierarchy
    stops when the smallest axis has 3 nodes (the 65^3 example coarsens to
    3x3x3).  Coordinates default to the node index (results do not depend on
    the scale or origin of the coordinates).
    """

    def __init__(self, dims, coords=None):
        dims = tuple(int(n) for n in dims)
        if not 1 <= len(dims) or any(n < 3 for n in dims):
            raise ValueError(f"every axis needs at least 3 nodes, got {dims}")
        self.ndim = len(dims)
        shapes = [dims]
        while min(shapes[-1]) > 3:
            shapes.append(tuple(len(coarse_indices(n)) for n in shapes[-1]))
        self.L = len(shapes) - 1
        self.levels = {self.L - i: s for i, s in enumerate(shapes)}
        if coords is None:
            coords = [None] * self.ndim
        xs = []
        for d, n in enumerate(dims):
            x = (np.arange(n, dtype=np.float64) if coords[d] is None
                 else np.asarray(coords[d], dtype=np.float64))
            if x.shape != (n,):
                raise ValueError(f"axis {d}: expected {n} coordinates")
            if not np.all(np.diff(x) > 0):
                raise ValueError(f"axis {d}: coordinates must increase strictly")
            xs.append(x)
        self.index = {self.L: [np.arange(n, dtype=np.int64) for n in dims]}
        for l in range(self.L, 0, -1):
            self.index[l - 1] = [ix[coarse_indices(len(ix))] for ix in self.index[l]]
        self.coords = {l: [xs[d][self.index[l][d]] for d in range(self.ndim)]
                       for l in range(self.L + 1)}
        self._ops = {}

    def ops(self, l: int) -> list[AxisOps]:
        """Per-axis operators of the level l -> l-1 transition."""
        if l not in self._ops:
            out = []
            for d in range(self.ndim):
                x = self.coords[l][d]
                keep = coarse_indices(len(x))
                out.append(AxisOps(keep, mass_matrix(x), prolongation(x, keep),
                                   mass_matrix(x[keep])))
            self._ops[l] = out
        return self._ops[l]

    def nodal_mask(self, l: int) -> np.ndarray:
        """Boolean array over ``N_l``: True on the nodes of ``N_{l-1}``."""
        m = np.zeros(self.levels[l], dtype=bool)
        m[np.ix_(*[o.keep for o in self.ops(l)])] = True
        return m


# --------------------------------------------------------------------------
# 1D finite-element operators
# --------------------------------------------------------------------------

def mass_matrix(x: np.ndarray) -> sp.csr_matrix:
    """P1 mass matrix ``M[i, j] = integral of phi_i phi_j`` on the nodes ``x``.

    On a cell of length ``D`` the two hat functions give ``D/3`` on the
    diagonal and ``D/6`` off it, so row ``j`` has diagonal
    ``(D_{j-1} + D_j) / 3`` and neighbours ``D_{j-1}/6``, ``D_j/6``.  For a
    uniform coarse grid of spacing ``2h`` this is the matrix printed in
    Section 5.4 (``2h/3`` at the ends, ``4h/3`` inside, ``h/3`` off the
    diagonal).
    """
    D = np.diff(np.asarray(x, dtype=np.float64))
    diag = np.zeros(len(x))
    diag[:-1] += D / 3.0
    diag[1:] += D / 3.0
    off = D / 6.0
    return sp.diags([off, diag, off], [-1, 0, 1], format="csr")


def prolongation(x: np.ndarray, keep: np.ndarray) -> sp.csr_matrix:
    """Piecewise-linear interpolation from the nodes ``x[keep]`` to all of
    ``x`` (``n x n'``).  Kept nodes copy their value; a node between kept
    nodes ``a < j < b`` takes ``(x_b - x_j)/(x_b - x_a)`` of the left value and
    ``(x_j - x_a)/(x_b - x_a)`` of the right one (Section 2, ``Pi_l``)."""
    x = np.asarray(x, dtype=np.float64)
    n, nc = len(x), len(keep)
    rows, cols, vals = [], [], []
    for k, j in enumerate(keep):
        rows.append(j); cols.append(k); vals.append(1.0)
    for k in range(nc - 1):
        a, b = int(keep[k]), int(keep[k + 1])
        for j in range(a + 1, b):
            rows += [j, j]
            cols += [k, k + 1]
            vals += [(x[b] - x[j]) / (x[b] - x[a]), (x[j] - x[a]) / (x[b] - x[a])]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))


def _banded(M: sp.spmatrix) -> np.ndarray:
    """Tridiagonal matrix in LAPACK banded storage (upper, main, lower)."""
    n = M.shape[0]
    ab = np.zeros((3, n))
    ab[1] = M.diagonal(0)
    if n > 1:
        ab[0, 1:] = M.diagonal(1)
        ab[2, :-1] = M.diagonal(-1)
    return ab


def project_axis(v: np.ndarray, axis: int, op: AxisOps) -> np.ndarray:
    """Apply ``A = M_c^{-1} P^T M_f`` along one axis: the 1D L2 projection
    (mass multiply, restriction to the load vector, tridiagonal solve;
    Section 2 step 4 and Section 5.2-5.4)."""
    vm = np.moveaxis(v, axis, 0)
    shape = vm.shape
    X = np.ascontiguousarray(vm).reshape(shape[0], -1)
    F = op.P.T @ (op.Mf @ X)
    Z = solve_banded((1, 1), _banded(op.Mc), F)
    return np.moveaxis(Z.reshape((op.Mc.shape[0],) + shape[1:]), 0, axis)


def project(v: np.ndarray, H: Hierarchy, l: int) -> np.ndarray:
    """``Q_{l-1}`` of a level-l nodal array: the tensor product of the 1D
    projections, applied axis by axis, axis d-1 first ("row sweep then
    column sweep", Section 5.1; the order does not matter in exact
    arithmetic)."""
    ops = H.ops(l)
    out = np.asarray(v, dtype=np.float64)
    for d in reversed(range(H.ndim)):
        out = project_axis(out, d, ops[d])
    return out


def interpolate(c: np.ndarray, H: Hierarchy, l: int) -> np.ndarray:
    """``Pi_{l-1}``: multilinear interpolation of level-(l-1) nodal values to
    all of ``N_l`` (tensor product of the 1D prolongations)."""
    out = np.asarray(c, dtype=np.float64)
    for d, op in enumerate(H.ops(l)):
        vm = np.moveaxis(out, d, 0)
        shape = vm.shape
        X = np.ascontiguousarray(vm).reshape(shape[0], -1)
        out = np.moveaxis((op.P @ X).reshape((op.P.shape[0],) + shape[1:]), 0, d)
    return out


# --------------------------------------------------------------------------
# Decomposition / recomposition (Section 2)
# --------------------------------------------------------------------------

def _check_stop(H: Hierarchy, stop_level: int):
    if not 0 <= stop_level <= H.L:
        raise ValueError(f"stop level {stop_level} outside [0, {H.L}]")


def decompose(u: np.ndarray, H: Hierarchy, stop_level: int = 0) -> np.ndarray:
    """Multilevel coefficients ``u_mc`` of ``u`` (Section 2).

    For ``l = L .. l~+1``: ``Q_{l-1}u`` is the projection of ``Q_l u``; the
    coefficients ``(I - Pi_{l-1}) Q_l u`` are stored at the nodes of
    ``N*_l``; the nodes of ``N_{l~}`` finally hold ``Q_{l~} u``.  ``u_mc`` is
    indexed by the finest grid, as Section 2 defines it."""
    _check_stop(H, stop_level)
    v = np.asarray(u, dtype=np.float64)
    if v.shape != H.levels[H.L]:
        raise ValueError("array shape does not match the hierarchy")
    out = v.copy()
    for l in range(H.L, stop_level, -1):
        keep = [o.keep for o in H.ops(l)]
        c = project(v, H, l)
        mc = v - interpolate(v[np.ix_(*keep)], H, l)
        out[np.ix_(*H.index[l])] = mc          # nodal entries are overwritten below
        v = c
    out[np.ix_(*H.index[stop_level])] = v
    return out


def recompose(umc: np.ndarray, H: Hierarchy, stop_level: int = 0) -> np.ndarray:
    """Inverse of :func:`decompose` (Section 2, recomposition steps 1-5).

    For ``l = l~+1 .. L``: ``z = Q_{l-1} w`` with ``w`` the level-l
    coefficients (zero on ``N_{l-1}``), ``Pi_{l-1}Q_l u = Q_{l-1}u - z`` on the
    coarse nodes, then ``Q_l u = Pi_{l-1}(Q_{l-1}u - z) + w``."""
    _check_stop(H, stop_level)
    umc = np.asarray(umc, dtype=np.float64)
    v = umc[np.ix_(*H.index[stop_level])].copy()
    for l in range(stop_level + 1, H.L + 1):
        w = umc[np.ix_(*H.index[l])].copy()
        w[H.nodal_mask(l)] = 0.0
        z = project(w, H, l)
        v = interpolate(v - z, H, l) + w
    return v


# --------------------------------------------------------------------------
# Level-wise quantization (Section 4.1, Algorithm 1)
# --------------------------------------------------------------------------

def projection_matrix(op: AxisOps) -> np.ndarray:
    """Dense ``A = M_c^{-1} P^T M_f`` (n' x n) of one axis."""
    R = (op.P.T @ op.Mf).toarray()
    return np.linalg.solve(op.Mc.toarray(), R)


def linf_constant(H: Hierarchy, stop_level: int = 0) -> float:
    """``C_Linf`` of Eq. (LInfNormEstimator) for this hierarchy.

    The paper takes the constant from its reference [ainsworth2019] without
    giving a value.  Reading used here, derived from the recomposition steps:
    with ``E_l`` the max-norm error of ``Q_l u`` and ``e_l`` that of the
    level-l coefficients, recomposition gives
    ``|E_l| <= |E_{l-1}| + (1 + |K_l|) |e_l|`` where ``K_l`` maps the level-l
    coefficients to the correction (interpolation has convex weights, so it
    does not enlarge the max norm).  Hence
    ``C = 1 + max_l |K_l|_inf`` makes ``sum_l tau_l <= tau / C`` sufficient.
    ``|K_l|_inf`` is the largest row sum over coarse rows of
    ``prod_d r_d - prod_d s_d`` where ``r_d`` / ``s_d`` are the absolute row
    sums of ``A_d`` over all / over coarse columns.  It is bounded from above
    by the telescoping sum
    ``sum_d (prod_{e<d} max s_e) max(r_d - s_d) (prod_{e>d} max r_e)``,
    which is what is used (exact in 1D; a valid upper bound in 2D/3D).
    ``C = 1`` when no level is decomposed.
    """
    _check_stop(H, stop_level)
    C = 1.0
    for l in range(stop_level + 1, H.L + 1):
        R, S, Dm = [], [], []
        for op in H.ops(l):
            A = np.abs(projection_matrix(op))
            r = A.sum(axis=1)
            s = A[:, op.keep].sum(axis=1)
            R.append(r.max()); S.append(s.max()); Dm.append((r - s).max())
        norm = 0.0
        for d in range(H.ndim):
            term = Dm[d]
            for e in range(d):
                term *= S[e]
            for e in range(d + 1, H.ndim):
                term *= R[e]
            norm += term
        C = max(C, 1.0 + norm)
    return C


def level_tolerances(H: Hierarchy, stop_level: int, tau: float,
                     C: float | None = None) -> np.ndarray:
    """Per-level tolerances ``tau_l`` for ``l = 0..L`` (entries below the
    stopping level are unused and set to ``tau_{l~}``).

    Algorithm 1 sets the stopping level's tolerance first and scales it by
    ``kappa = sqrt(2^d)`` per finer level (Eq. (LinfTau) with the sum starting at
    the stopping level), so that ``sum_{l>=l~} tau_l = tau / C``."""
    _check_stop(H, stop_level)
    if C is None:
        C = linf_constant(H, stop_level)
    kappa = math.sqrt(2.0 ** H.ndim)
    m = H.L + 1 - stop_level
    kpow = 1.0
    for _ in range(m):
        kpow *= kappa
    taus = np.empty(H.L + 1)
    taus[stop_level] = (1.0 - kappa) * tau / ((1.0 - kpow) * C)
    for l in range(stop_level + 1, H.L + 1):
        taus[l] = kappa * taus[l - 1]
    taus[:stop_level] = taus[stop_level]
    return taus


def node_levels(H: Hierarchy, stop_level: int = 0) -> np.ndarray:
    """Level of every finest node: the least ``l`` with the node in ``N_l``
    (Section 2's indexing of ``u_mc``), raised to the stopping level because
    the whole of ``N_{l~}`` is quantized with ``tau_{l~}`` (as Algorithm 1
    does)."""
    per_axis = []
    for d in range(H.ndim):
        lev = np.full(H.levels[H.L][d], H.L, dtype=np.int64)
        for l in range(H.L - 1, -1, -1):
            lev[H.index[l][d]] = l
        per_axis.append(lev)
    out = per_axis[0]
    for lev in per_axis[1:]:
        out = np.maximum.outer(out, lev)
    return np.maximum(out.reshape(H.levels[H.L]), stop_level)


def llround(y: np.ndarray) -> np.ndarray:
    """Round to the nearest integer, ties away from zero, exactly: the
    fractional part ``y - trunc(y)`` is exact in binary floating point."""
    y = np.asarray(y, dtype=np.float64)
    t = np.trunc(y)
    return (t + np.sign(y) * (np.abs(y - t) >= 0.5)).astype(np.int64)


def quantize(umc: np.ndarray, H: Hierarchy, stop_level: int,
             taus: np.ndarray) -> np.ndarray:
    """Labels ``round(u_mc / q_l)`` with bin width ``q_l = 2 tau_l`` and the
    bin centre as the value (Section 4.1), computed in FP64 (an FP32
    coefficient is widened first)."""
    lev = node_levels(H, stop_level)
    q = 2.0 * np.asarray(taus, dtype=np.float64)[lev]
    return llround(np.asarray(umc, dtype=np.float64) / q)


def dequantize(labels: np.ndarray, H: Hierarchy, stop_level: int,
               taus: np.ndarray, dtype=np.float64) -> np.ndarray:
    """Bin centres ``label * q_l`` in FP64, rounded to ``dtype``."""
    lev = node_levels(H, stop_level)
    q = 2.0 * np.asarray(taus, dtype=np.float64)[lev]
    return (np.asarray(labels, dtype=np.int64).astype(np.float64) * q).astype(dtype)


def value_range(u: np.ndarray) -> float:
    """``max u - min u`` in FP64: the scale of a relative error bound."""
    u = np.asarray(u, dtype=np.float64)
    return float(u.max() - u.min())


# --------------------------------------------------------------------------
# Adaptive stopping level (Section 4.2, Algorithm 1's stopping-level search)
# --------------------------------------------------------------------------

# Penalty factors, in units of the level's tolerance tau_0 (Section 4.2): the
# 3D Lorenzo predictor (Eq. (lorenzo)) and multilinear interpolation at edge,
# plane and cube nodes (Eq. (interp)), keyed by the number of axes along
# which the node is a cell midpoint.  The paper derives them for 3D only.
LORENZO_PENALTY = 1.22
INTERP_PENALTY = {1: 0.369, 2: 0.259, 3: 0.182}


def sampled_blocks(H: Hierarchy, l: int):
    """The sampled ``3^d`` blocks of the level-l grid (Section 4.2): a block
    is a cell of the level-(l-1) grid, spanning level-l indices
    ``keep[b] .. keep[b+1]`` on every axis (3 nodes, or 2 for the last cell
    of an even axis); one cell in four is taken along each axis (``b`` a
    multiple of 4).  Returns per-axis lists of (first, last) index pairs."""
    out = []
    for op in H.ops(l):
        keep = op.keep
        out.append([(int(keep[b]), int(keep[b + 1])) for b in range(0, len(keep) - 1, 4)])
    return out


def _lorenzo(v: np.ndarray, idx) -> float:
    """Lorenzo prediction at ``idx`` (Eq. (lorenzo)): the signed sum over the
    2^d - 1 neighbours with some indices decreased by one, ``+`` for an odd
    number of decreased indices; neighbours outside the grid count as 0."""
    d = v.ndim
    pred = 0.0
    for mask in range(1, 1 << d):
        nb = list(idx)
        inside = True
        for a in range(d):
            if mask >> a & 1:
                nb[a] -= 1
                inside = inside and nb[a] >= 0
        if inside:
            sign = 1.0 if bin(mask).count("1") % 2 == 1 else -1.0
            pred += sign * float(v[tuple(nb)])
    return pred


def prediction_errors(v: np.ndarray, H: Hierarchy, l: int, tau0: float):
    """``(E_Lorenzo, E_interp)``, Algorithm 1's sampled prediction errors, for
    the level-l grid ``v``: over every coefficient node (a node outside ``N_{l-1}``) of
    the sampled blocks, ``|Lorenzo prediction - v| + 1.22 tau0`` and
    ``|Pi_{l-1} v - v| + p tau0`` with ``p`` the edge / plane / cube penalty
    of the node (Eqs. (lorenzo), (interp)).  Interpolation uses the grid's
    own coordinates (the uniform-grid stencils of Eq. (multilinear_interp)
    are its special case).  Sums run over the blocks in C order and over the
    nodes of a block in C order.  3D only."""
    if H.ndim != 3:
        raise ValueError("the penalty factors of Section 4.2 are for 3D grids")
    v = np.asarray(v, dtype=np.float64)
    if v.shape != H.levels[l]:
        raise ValueError("array shape does not match level l")
    keep = [o.keep for o in H.ops(l)]
    pred_i = interpolate(v[np.ix_(*keep)], H, l)
    is_nodal = [np.isin(np.arange(n), k) for n, k in zip(v.shape, keep)]
    blocks = sampled_blocks(H, l)
    e_lor = 0.0
    e_int = 0.0
    for b0 in blocks[0]:
        for b1 in blocks[1]:
            for b2 in blocks[2]:
                for i in range(b0[0], b0[1] + 1):
                    for j in range(b1[0], b1[1] + 1):
                        for k in range(b2[0], b2[1] + 1):
                            mids = (int(not is_nodal[0][i]) + int(not is_nodal[1][j]) +
                                    int(not is_nodal[2][k]))
                            if mids == 0:
                                continue
                            x = float(v[i, j, k])
                            e_lor += abs(_lorenzo(v, (i, j, k)) - x) + LORENZO_PENALTY * tau0
                            e_int += abs(float(pred_i[i, j, k]) - x) + INTERP_PENALTY[mids] * tau0
    return e_lor, e_int


def adaptive_stop_level(u: np.ndarray, H: Hierarchy, tau: float):
    """Algorithm 1's stopping-level search: for ``l = L, L-1, ..``, with ``tau_0`` the
    tolerance of level ``l`` were it the stopping level, sample
    ``Q_l u`` and stop at ``l`` when the Lorenzo estimate is below the
    interpolation estimate; otherwise project to ``Q_{l-1} u`` and go on.
    Reading: the loop ends at level 1 (a level-0 grid has no coarser grid to
    interpolate from), so the stopping level is 0 when no level stops it.
    Returns the stopping level and ``{l: (E_Lorenzo, E_interp)}`` for every
    sampled level."""
    v = np.asarray(u, dtype=np.float64)
    sums = {}
    for l in range(H.L, 0, -1):
        tau0 = float(level_tolerances(H, l, tau)[l])
        e = prediction_errors(v, H, l, tau0)
        sums[l] = e
        if e[0] < e[1]:
            return l, sums
        v = project(v, H, l)
    return 0, sums


# --------------------------------------------------------------------------
# Progressive recomposition and iso-surface area (Section 1; Section 6.2.2)
# --------------------------------------------------------------------------

def recompose_partial(umc: np.ndarray, H: Hierarchy, stop_level: int, level: int) -> np.ndarray:
    """``Q_k u`` on the level-k grid from the decomposed array ``umc``
    (stopping level ``stop_level`` <= k = ``level`` <= L): the refactored
    reconstruction of reduced size that Section 1 describes, obtained by
    summing the components of levels ``stop_level .. k`` only, i.e. the
    recomposition of the levels up to k (Section 2's recomposition,
    stopped at level k)."""
    _check_stop(H, stop_level)
    if not stop_level <= level <= H.L:
        raise ValueError("target level outside [stop level, L]")
    umc = np.asarray(umc, dtype=np.float64)
    v = umc[np.ix_(*H.index[stop_level])].copy()
    for l in range(stop_level + 1, level + 1):
        w = umc[np.ix_(*H.index[l])].copy()
        w[H.nodal_mask(l)] = 0.0
        z = project(w, H, l)
        v = interpolate(v - z, H, l) + w
    return v


# The 6 tetrahedra of a cell around its main diagonal (corner 0 to corner 7);
# corner c has offsets ((c >> 2) & 1, (c >> 1) & 1, c & 1) along axes 0, 1, 2.
TETS = ((0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7))


def _tri_area(a, b, c) -> float:
    return 0.5 * float(np.linalg.norm(np.cross(np.subtract(b, a), np.subtract(c, a))))


def _tet_area(p, f, iso) -> float:
    """Area of the piece of the iso-surface f = iso inside one tetrahedron
    with vertex positions ``p`` and values ``f`` (f linear in the
    tetrahedron).  A vertex is above when f > iso.  The surface crosses each
    edge joining an above and a below vertex at the linear interpolant's
    root; one vertex apart gives a triangle, two apart a quadrilateral,
    split along the diagonal from the (below 0, above 0) edge point to the
    (below 1, above 1) one."""
    up = [i for i in range(4) if f[i] > iso]
    dn = [i for i in range(4) if not f[i] > iso]
    if not up or not dn:
        return 0.0

    def cross(a, b):
        t = (iso - f[a]) / (f[b] - f[a])
        return tuple(p[a][d] + t * (p[b][d] - p[a][d]) for d in range(3))

    if len(up) == 1 or len(dn) == 1:
        one, rest = (up[0], dn) if len(up) == 1 else (dn[0], up)
        return _tri_area(*[cross(one, r) for r in rest])
    a, b = dn
    c, d = up
    q0, q1, q2, q3 = cross(a, c), cross(a, d), cross(b, d), cross(b, c)
    return _tri_area(q0, q1, q2) + _tri_area(q0, q2, q3)


def iso_area(v: np.ndarray, coords, iso: float) -> float:
    """Area of the iso-surface ``v = iso`` of the 3D grid function ``v`` with
    axis coordinates ``coords`` (None: the node index), the analysis of the
    use case in Section 6.2.2.  The paper names the quantity, not the
    method; here every cell is split into the 6 tetrahedra around its main
    diagonal and ``v`` is taken linear on each (marching tetrahedra), which
    reproduces planar iso-surfaces exactly.  Cells are visited in C order;
    the sum is in FP64."""
    v = np.asarray(v, dtype=np.float64)
    if v.ndim != 3:
        raise ValueError("iso-surface area is defined for 3D grids")
    xs = [np.arange(n, dtype=np.float64) if (coords is None or coords[d] is None)
          else np.asarray(coords[d], dtype=np.float64) for d, n in enumerate(v.shape)]
    total = 0.0
    n0, n1, n2 = v.shape
    for i in range(n0 - 1):
        for j in range(n1 - 1):
            for k in range(n2 - 1):
                cf = [float(v[i + (c >> 2 & 1), j + (c >> 1 & 1), k + (c & 1)]) for c in range(8)]
                if min(cf) > iso or max(cf) <= iso:
                    continue
                cp = [(xs[0][i + (c >> 2 & 1)], xs[1][j + (c >> 1 & 1)], xs[2][k + (c & 1)])
                      for c in range(8)]
                for t in TETS:
                    total += _tet_area([cp[c] for c in t], [cf[c] for c in t], iso)
    return total


# --------------------------------------------------------------------------
# Lossless stage for the labels (Section 4.1, the last step of Algorithm 1)
# and PSNR
# (Section 6, "Quality")
# --------------------------------------------------------------------------

PACK_CHUNK = 1024


def _zigzag(k: int) -> int:
    """Signed to unsigned, small magnitudes to small codes: 0, -1, 1, -2, ..
    map to 0, 1, 2, 3, .."""
    return (k << 1) if k >= 0 else ((-k) << 1) - 1


def pack_labels(labels) -> bytes:
    """The labels' lossless stream.  The paper passes the labels to a
    general-purpose lossless coder; this library's coder (a reading) packs
    them in chunks of 1024: each label is zigzag-coded and stored in the
    chunk's width w, the bit length of the chunk's largest code (0 when all
    are 0), least significant bit first, in little-endian 64-bit words.
    Layout: uint64 N | one width byte per chunk | zero padding to 8 bytes |
    for each chunk, ceil(n_c w / 64) words."""
    k = [int(v) for v in np.asarray(labels, dtype=np.int64).ravel()]
    n = len(k)
    chunks = [k[i:i + PACK_CHUNK] for i in range(0, n, PACK_CHUNK)]
    widths = [max((_zigzag(v) for v in c), default=0).bit_length() for c in chunks]
    out = bytearray(n.to_bytes(8, "little"))
    out += bytes(widths)
    out += bytes((-len(out)) % 8)
    for c, w in zip(chunks, widths):
        bits = 0
        for i, v in enumerate(c):
            bits |= _zigzag(v) << (i * w)
        nwords = (len(c) * w + 63) // 64
        out += bits.to_bytes(8 * nwords, "little")
    return bytes(out)


def unpack_labels(buf: bytes) -> np.ndarray:
    """Inverse of :func:`pack_labels`."""
    buf = bytes(buf)
    n = int.from_bytes(buf[:8], "little")
    nchunks = (n + PACK_CHUNK - 1) // PACK_CHUNK
    widths = list(buf[8:8 + nchunks])
    off = 8 + nchunks
    off += (-off) % 8
    out = []
    for c, w in enumerate(widths):
        nc = min(PACK_CHUNK, n - c * PACK_CHUNK)
        nwords = (nc * w + 63) // 64
        bits = int.from_bytes(buf[off:off + 8 * nwords], "little")
        off += 8 * nwords
        mask = (1 << w) - 1
        for i in range(nc):
            z = (bits >> (i * w)) & mask
            out.append((z >> 1) if z % 2 == 0 else -((z + 1) >> 1))
    return np.asarray(out, dtype=np.int64)


def psnr(u: np.ndarray, v: np.ndarray) -> float:
    """PSNR of a reconstruction ``v`` of ``u`` (Section 6, "Quality"): the
    printed formula's range term is garbled (max u - min v); the value range
    of the original, max u - min u, is used, in FP64."""
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    mse = float(np.mean((u - v) ** 2))
    return 20.0 * math.log10(float(u.max() - u.min())) - 10.0 * math.log10(mse)


# --------------------------------------------------------------------------
# Other bin-width rules (Section 4.1): L-inf-optimal widths and L2 control
# --------------------------------------------------------------------------

def _level_counts(H: Hierarchy, stop_level: int) -> np.ndarray:
    """#N*_l for l = 0..L: the nodes new at level l, with the whole coarse
    block N_{l~} counted at the stopping level (it is quantized with
    tau_{l~}); 0 below the stopping level."""
    n = [int(np.prod(H.levels[l])) for l in range(H.L + 1)]
    out = np.zeros(H.L + 1)
    out[stop_level] = n[stop_level]
    for l in range(stop_level + 1, H.L + 1):
        out[l] = n[l] - n[l - 1]
    return out


def _cell_measure(H: Hierarchy, l: int) -> float:
    """``h_l^d``: the product over the axes of the largest row sum of the
    level-l 1D mass matrix (the integral of a hat function), which equals
    h^d on a uniform grid of spacing h and bounds the mass matrix's largest
    eigenvalue on any grid."""
    out = 1.0
    for d in range(H.ndim):
        M = mass_matrix(H.coords[l][d])
        out *= float(np.max(np.asarray(M.sum(axis=1)).ravel()))
    return out


def level_tolerances_mode(H: Hierarchy, stop_level: int, tau: float, mode: str) -> np.ndarray:
    """Per-level tolerances ``tau_l`` (l = 0..L; below the stopping level
    they repeat tau_{l~}) for the three rules of Section 4.1:

    * ``"geometric"``: Eq. (LinfTau), ``tau_l = kappa^(l-l~) tau_{l~}`` with
      ``sum tau_l = tau / C_Linf`` (the rule used throughout);
    * ``"linf_optimal"``: the widths that minimise the estimated label cost
      under the same L-infinity condition, ``tau_l = tau / C_Linf * #N*_l /
      #N_L`` (noted in Section 4.1 for completeness);
    * ``"l2"``: ``tau`` bounds the L2 norm of the reconstruction error:
      ``tau_l = tau / (C_L2 h_l^d #N_L)^(1/2)``, which meets
      ``sum_l h_l^d #N*_l tau_l^2 = tau^2 / C_L2``.  Reading: C_L2 = 1 with
      h_l^d the largest mass-matrix row-sum product of level l; the
      multilevel error components (I - Q_{l-1}) e_l are L2-orthogonal and
      each is at most its nodal P1 function's norm, at most h_l^d sum e^2,
      so the bound holds with that constant."""
    if mode == "geometric":
        return level_tolerances(H, stop_level, tau)
    _check_stop(H, stop_level)
    cnt = _level_counts(H, stop_level)
    nL = float(np.prod(H.levels[H.L]))
    taus = np.empty(H.L + 1)
    if mode == "linf_optimal":
        C = linf_constant(H, stop_level)
        for l in range(stop_level, H.L + 1):
            taus[l] = tau / C * cnt[l] / nL
    elif mode == "l2":
        for l in range(stop_level, H.L + 1):
            taus[l] = tau / math.sqrt(_cell_measure(H, l) * nL)
    else:
        raise ValueError(f"unknown mode {mode}")
    taus[:stop_level] = taus[stop_level]
    return taus


def l2_error(e: np.ndarray, H: Hierarchy) -> float:
    """L2 norm of the P1 function with nodal values ``e`` on the finest
    grid: sqrt(e^T M e), M the tensor-product mass matrix."""
    e = np.asarray(e, dtype=np.float64)
    Me = e
    for d in range(H.ndim):
        M = mass_matrix(H.coords[H.L][d])
        vm = np.moveaxis(Me, d, 0)
        shape = vm.shape
        X = np.ascontiguousarray(vm).reshape(shape[0], -1)
        Me = np.moveaxis((M @ X).reshape(shape), 0, d)
    return math.sqrt(float(np.sum(e * Me)))


# --------------------------------------------------------------------------
# Coarse-part predictor (the coarse part's coder in Algorithm 1; Section 4.2,
# Eq. (lorenzo))
# --------------------------------------------------------------------------

def _coarse_block(labels, H: Hierarchy, stop_level: int):
    return np.ix_(*H.index[stop_level])


def lorenzo_encode(labels: np.ndarray, H: Hierarchy, stop_level: int) -> np.ndarray:
    """Labels with the coarse block N_{l~} replaced by its Lorenzo residuals:
    r = q - pred(q), pred the signed sum of the 2^d - 1 lower neighbours in
    the coarse grid (0 outside it), in 64-bit wrap-around integer arithmetic
    (an exact bijection).  The coarse labels are the linear quantization of
    Q_{l~}u with bin 2 tau_{l~}, so predicting from them is predicting from
    the reconstructed values, as the Lorenzo coder of Section 4.2 does; the
    residuals of a smooth coarse part are small and pack tightly."""
    out = np.array(labels, dtype=np.int64, copy=True)
    ix = _coarse_block(out, H, stop_level)
    q = out[ix].astype(np.uint64)
    r = q.copy()
    d = q.ndim
    for mask in range(1, 1 << d):
        shifted = q
        for a in range(d):
            if mask >> a & 1:
                pad = [(0, 0)] * d
                pad[a] = (1, 0)
                shifted = np.pad(shifted, pad)[tuple(slice(0, n) for n in q.shape)]
        if bin(mask).count("1") % 2 == 1:
            r = r - shifted
        else:
            r = r + shifted
    out[ix] = r.astype(np.int64)
    return out


def lorenzo_decode(labels: np.ndarray, H: Hierarchy, stop_level: int) -> np.ndarray:
    """Inverse of :func:`lorenzo_encode`: the residual operator is the product
    of the backward differences along every axis, so cumulative sums along
    every axis (64-bit wrap-around) restore the labels."""
    out = np.array(labels, dtype=np.int64, copy=True)
    ix = _coarse_block(out, H, stop_level)
    q = out[ix].astype(np.uint64)
    for a in range(q.ndim):
        q = np.cumsum(q, axis=a, dtype=np.uint64)
    out[ix] = q.astype(np.int64)
    return out


# --------------------------------------------------------------------------
# Entropy of the labels and the cost model (Section 4.1), and a canonical
# Huffman coder of the labels (a reading of Algorithm 1's final lossless
# encoder)
# --------------------------------------------------------------------------

def label_entropy(labels) -> float:
    """Order-0 Shannon entropy of the labels in bits per label (Section 4.1
    estimates the encoding cost with it): ``-sum_v p_v log2 p_v`` over the
    distinct values, ``p_v`` their relative counts; 0 for no labels."""
    k = np.asarray(labels, dtype=np.int64).ravel()
    if k.size == 0:
        return 0.0
    _, cnt = np.unique(k, return_counts=True)
    p = cnt.astype(np.float64) / k.size
    return float(-(p * np.log2(p)).sum())


def cost_model(H: Hierarchy, stop_level: int, taus, R: float) -> float:
    """Estimated cost in bits of the level-wise labels, Section 4.1:
    ``sum_l #N*_l log2(R / q_l)`` with ``q_l = 2 tau_l`` and R the range of
    the multilevel coefficients (the coarse block N_{l~} counted at the
    stopping level, as it is quantized with tau_{l~})."""
    cnt = _level_counts(H, stop_level)
    taus = np.asarray(taus, dtype=np.float64)
    return float(sum(cnt[l] * math.log2(R / (2.0 * taus[l]))
                     for l in range(stop_level, H.L + 1)))


HUFF_CHUNK = 1024
HUFF_DIRECT = 32768     # zigzag codes below this are symbols of their own
HUFF_K = HUFF_DIRECT + 49   # then one symbol per bit length 16 .. 64
HUFF_MAXLEN = 31


def huffman_lengths(counts) -> list:
    """Code lengths of a Huffman code for symbol counts (0 = unused symbol).

    Huffman's construction with a fixed order, so that the lengths are a
    function of the counts alone: leaves sorted by (count, symbol), merged
    nodes queued in the order they are made; each step takes the lighter of
    the two queue heads, a leaf on a tie.  One used symbol gets length 1.  If
    the longest code exceeds 31 bits, every used count c becomes
    max(1, c // 2) and the code is rebuilt (a reading: the paper's coder has
    no length limit; this keeps every code in 32 bits)."""
    counts = [int(c) for c in counts]
    while True:
        used = sorted((c, s) for s, c in enumerate(counts) if c > 0)
        lengths = [0] * len(counts)
        if not used:
            return lengths
        if len(used) == 1:
            lengths[used[0][1]] = 1
            return lengths
        parent = {}
        leaves = [(c, ("leaf", s)) for c, s in used]
        merged = []
        li = mi = 0
        nid = 0

        def take():
            nonlocal li, mi
            if mi >= len(merged) or (li < len(leaves) and leaves[li][0] <= merged[mi][0]):
                li += 1
                return leaves[li - 1]
            mi += 1
            return merged[mi - 1]

        while (len(leaves) - li) + (len(merged) - mi) > 1:
            a = take()
            b = take()
            node = ("node", nid)
            nid += 1
            parent[a[1]] = node
            parent[b[1]] = node
            merged.append((a[0] + b[0], node))
        for _, s in used:
            d, x = 0, ("leaf", s)
            while x in parent:
                x = parent[x]
                d += 1
            lengths[s] = d
        if max(lengths) <= HUFF_MAXLEN:
            return lengths
        counts = [max(1, c // 2) if c > 0 else 0 for c in counts]


def huffman_codes(lengths) -> dict:
    """Canonical codes: symbols ordered by (length, symbol) take consecutive
    code values, the first of each length being (first of the previous
    length + its count) shifted left by the length difference."""
    order = sorted((L, s) for s, L in enumerate(lengths) if L > 0)
    codes, code, prev = {}, 0, None
    for L, s in order:
        if prev is not None:
            code = (code + 1) << (L - prev)
        codes[s] = code
        prev = L
    return codes


def _huff_symbol(z: int):
    """(symbol, extra bits, number of extra bits) of a zigzag code: codes
    below 2^15 are their own symbol; a larger code of bit length b is the
    symbol 32768 + b - 16 followed by its b - 1 low bits (its leading 1 is
    implied), as DEFLATE codes lengths with extra bits."""
    if z < HUFF_DIRECT:
        return z, 0, 0
    b = z.bit_length()
    return HUFF_DIRECT + b - 16, z - (1 << (b - 1)), b - 1


def huffman_encode(labels) -> bytes:
    """The labels' Huffman stream.  Layout (little-endian): uint64 N |
    uint32 K (32817) | uint32 longest code length | K bytes of code lengths
    (0 = unused symbol) | zero padding to 8 bytes | per chunk of 1024 labels
    a uint32 word count | zero padding to 8 bytes | per chunk its 64-bit
    words.  Each label's
    symbol code is written most significant bit first at increasing bit
    positions from the least significant bit of the chunk's first word,
    followed by its extra bits, least significant first."""
    z = [_zigzag(int(v)) for v in np.asarray(labels, dtype=np.int64).ravel()]
    n = len(z)
    parts = [_huff_symbol(v) for v in z]
    counts = [0] * HUFF_K
    for s, _, _ in parts:
        counts[s] += 1
    lengths = huffman_lengths(counts)
    codes = huffman_codes(lengths)
    out = bytearray(n.to_bytes(8, "little"))
    out += HUFF_K.to_bytes(4, "little") + max(lengths).to_bytes(4, "little")
    out += bytes(lengths)
    out += bytes((-len(out)) % 8)
    payload = []
    for c0 in range(0, n, HUFF_CHUNK):
        bits, pos = 0, 0
        for s, extra, nx in parts[c0:c0 + HUFF_CHUNK]:
            L, code = lengths[s], codes[s]
            for i in range(L):
                bits |= ((code >> (L - 1 - i)) & 1) << (pos + i)
            pos += L
            bits |= extra << pos
            pos += nx
        nwords = (pos + 63) // 64
        out += nwords.to_bytes(4, "little")
        payload.append(bits.to_bytes(8 * nwords, "little"))
    out += bytes((-len(out)) % 8)
    for p in payload:
        out += p
    return bytes(out)


def huffman_decode(buf: bytes) -> np.ndarray:
    """Inverse of :func:`huffman_encode`: read code bits one at a time; a
    code of length L is complete when it falls among the canonical codes of
    that length; a bit-length symbol is followed by its extra bits."""
    buf = bytes(buf)
    n = int.from_bytes(buf[0:8], "little")
    K = int.from_bytes(buf[8:12], "little")
    lengths = list(buf[16:16 + K])
    codes = huffman_codes(lengths)
    lookup = {(lengths[s], c): s for s, c in codes.items()}
    nchunks = (n + HUFF_CHUNK - 1) // HUFF_CHUNK
    off = 16 + K
    off += (-off) % 8
    words = []
    for c in range(nchunks):
        words.append(int.from_bytes(buf[off:off + 4], "little"))
        off += 4
    off += (-off) % 8
    out = []
    for c in range(nchunks):
        bits = int.from_bytes(buf[off:off + 8 * words[c]], "little")
        off += 8 * words[c]
        pos = 0
        for _ in range(min(HUFF_CHUNK, n - c * HUFF_CHUNK)):
            code, L = 0, 0
            while True:
                code = (code << 1) | ((bits >> pos) & 1)
                pos += 1
                L += 1
                if (L, code) in lookup:
                    s = lookup[(L, code)]
                    break
            if s < HUFF_DIRECT:
                zv = s
            else:
                b = s - HUFF_DIRECT + 16
                zv = (1 << (b - 1)) | ((bits >> pos) & ((1 << (b - 1)) - 1))
                pos += b - 1
            out.append((zv >> 1) if zv % 2 == 0 else -((zv + 1) >> 1))
    return np.asarray(out, dtype=np.int64)
