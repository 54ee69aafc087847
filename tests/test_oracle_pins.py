"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here re-types an oracle formula: the expected values come from hand
derivations (tests/golden), numbers printed in the paper (Lemma 1, the mass
matrix of Section 5.4, the interpolation stencils of Section 4.2), numerical
quadrature with an independent piecewise-linear evaluator, exact rational
arithmetic, dense Kronecker brute force, and invariants of the transform.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import fields as F

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- golden ---

def _golden_cases():
    cases = []
    with open(os.path.join(GOLDEN, "corrections.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            dims_s, coords_s, w_s, exp_s = [p.strip() for p in line.split("|")]
            dims = tuple(int(v) for v in dims_s.split("x"))
            coords = []
            for c in coords_s.split(";"):
                coords.append(None if c == "u" else np.array([float(v) for v in c.split(",")]))
            w = np.zeros(dims)
            for ent in w_s.split():
                idx, val = ent.split(":")
                w[tuple(int(v) for v in idx.split(","))] = float(val)
            exp = np.array([float(Fraction(v)) for v in exp_s.split()])
            cases.append((dims, coords, w, exp))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: str(c[0]))
def test_golden_corrections(case):
    """Hand-derived exact corrections (Section 2 step 4)."""
    dims, coords, w, exp = case
    H = O.Hierarchy(dims, coords)
    z = O.project(w, H, H.L)
    np.testing.assert_allclose(z.ravel(), exp, rtol=0, atol=1e-15)


def test_golden_node_levels():
    with open(os.path.join(GOLDEN, "node_levels.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n_s, L_s, lev_s = [p.strip() for p in line.split("|")]
            H = O.Hierarchy((int(n_s),))
            assert H.L == int(L_s)
            assert O.node_levels(H).tolist() == [int(v) for v in lev_s.split()]


# ------------------------------------------------ printed paper numbers ---

def test_lemma1_interior_weights():
    """Lemma 1 (Section 5.2): interior load-vector row of P^T M_f on a
    uniform grid of spacing h is h (1/12, 1/2, 5/6, 1/2, 1/12)."""
    h = 0.37
    x = h * np.arange(17)
    keep = O.coarse_indices(17)
    R = (O.prolongation(x, keep).T @ O.mass_matrix(x)).toarray()
    for k in range(1, len(keep) - 1):
        row = R[k, 2 * k - 2: 2 * k + 3]
        np.testing.assert_allclose(row, h * np.array([1 / 12, 1 / 2, 5 / 6, 1 / 2, 1 / 12]),
                                   rtol=1e-14)
        assert np.count_nonzero(np.abs(R[k]) > 1e-300) == 5


def test_printed_coarse_mass_matrix():
    """Section 5.4: coarse mass matrix on a level with fine spacing h has
    2h/3 at the ends, 4h/3 inside and h/3 off the diagonal."""
    h = 0.25
    xc = 2 * h * np.arange(7)
    M = O.mass_matrix(xc).toarray()
    n = len(xc)
    for i in range(n):
        assert M[i, i] == pytest.approx((2 / 3 if i in (0, n - 1) else 4 / 3) * h, rel=1e-15)
        if i + 1 < n:
            assert M[i, i + 1] == pytest.approx(h / 3, rel=1e-15)
            assert M[i + 1, i] == pytest.approx(h / 3, rel=1e-15)


def test_interpolation_stencils():
    """Eq. (multilinear_interp), Section 4.2: edge, plane and cube nodes take
    1/2, 1/4 and 1/8 of the surrounding nodal values."""
    H = O.Hierarchy((5, 5, 5))
    c = _rng(1).standard_normal((3, 3, 3))
    v = O.interpolate(c, H, 1)
    u = {(2 * a, 2 * b, 2 * e): c[a, b, e] for a in range(2) for b in range(2) for e in range(2)}
    assert v[0, 0, 1] == pytest.approx(0.5 * (u[0, 0, 0] + u[0, 0, 2]), abs=1e-15)
    assert v[0, 1, 1] == pytest.approx(0.25 * (u[0, 0, 0] + u[0, 0, 2] + u[0, 2, 0] + u[0, 2, 2]),
                                       abs=1e-15)
    assert v[1, 1, 1] == pytest.approx(0.125 * sum(u.values()), abs=1e-15)
    for key in np.ndindex(3, 3, 3):
        assert v[tuple(2 * i for i in key)] == c[key]


# ------------------------------------------- quadrature orthogonality ---

def _gauss3():
    return np.polynomial.legendre.leggauss(3)


def _pl_eval_1d(xn, vals, xq):
    return np.interp(xq, xn, vals)


def test_projection_orthogonality_1d_quadrature():
    """The L2 projection is the coarse function whose error is orthogonal to
    every coarse hat function: integral (w_h - z_H) phi_k = 0.  Integrals by
    3-point Gauss-Legendre per fine cell (exact for products of linears),
    with functions evaluated by np.interp -- independent of the oracle's
    matrices."""
    rng = _rng(2)
    for n in (5, 8, 13, 24):
        x = np.sort(rng.uniform(0, 3, n))
        x[0], x[-1] = 0.0, 3.0
        w = rng.standard_normal(n)
        H = O.Hierarchy((n,), [x])
        z = O.project(w, H, H.L)
        xc = H.coords[H.L - 1][0]
        gx, gw = _gauss3()
        resid = np.zeros(len(xc))
        for a, b in zip(x[:-1], x[1:]):
            xq = 0.5 * (b - a) * gx + 0.5 * (a + b)
            wq = 0.5 * (b - a) * gw
            err = _pl_eval_1d(x, w, xq) - _pl_eval_1d(xc, z, xq)
            for k in range(len(xc)):
                e = np.zeros(len(xc)); e[k] = 1.0
                resid[k] += np.sum(wq * err * _pl_eval_1d(xc, e, xq))
        assert np.abs(resid).max() < 1e-13 * max(1.0, np.abs(w).max())


def test_projection_orthogonality_2d_quadrature():
    """2D version with a tensor Gauss rule per fine cell and bilinear
    evaluation by scipy's RegularGridInterpolator."""
    rng = _rng(3)
    dims = (6, 7)
    xs = []
    for n in dims:
        x = np.sort(rng.uniform(0, 1, n)); x[0], x[-1] = 0.0, 1.0
        xs.append(x)
    w = rng.standard_normal(dims)
    H = O.Hierarchy(dims, xs)
    z = O.project(w, H, H.L)
    xc = H.coords[H.L - 1]
    fw = RegularGridInterpolator(xs, w)
    fz = RegularGridInterpolator(xc, z)
    gx, gw = _gauss3()
    pts, wts = [], []
    for a0, b0 in zip(xs[0][:-1], xs[0][1:]):
        for a1, b1 in zip(xs[1][:-1], xs[1][1:]):
            q0 = 0.5 * (b0 - a0) * gx + 0.5 * (a0 + b0)
            q1 = 0.5 * (b1 - a1) * gx + 0.5 * (a1 + b1)
            P0, P1 = np.meshgrid(q0, q1, indexing="ij")
            W = np.outer(0.5 * (b0 - a0) * gw, 0.5 * (b1 - a1) * gw)
            pts.append(np.stack([P0.ravel(), P1.ravel()], 1)); wts.append(W.ravel())
    pts = np.concatenate(pts); wts = np.concatenate(wts)
    pts = np.clip(pts, [xs[0][0], xs[1][0]], [xs[0][-1], xs[1][-1]])
    err = fw(pts) - fz(pts)
    for k0 in range(len(xc[0])):
        for k1 in range(len(xc[1])):
            e = np.zeros((len(xc[0]), len(xc[1]))); e[k0, k1] = 1
            phi = RegularGridInterpolator(xc, e)(pts)
            assert abs(np.sum(wts * err * phi)) < 1e-13


def test_textbook_l2_projection_1d_continuous():
    """d = 1 reduces to the textbook P1 L2 projection: projecting the
    interpolant of a fine function and minimising the L2 error over coarse
    coefficients by least squares on dense quadrature samples gives the same
    coarse values (scipy lstsq on sampled hat functions)."""
    rng = _rng(4)
    n = 11
    x = np.sort(rng.uniform(0, 1, n)); x[0], x[-1] = 0, 1
    w = rng.standard_normal(n)
    H = O.Hierarchy((n,), [x])
    z = O.project(w, H, H.L)
    xc = H.coords[H.L - 1][0]
    gx, gw = _gauss3()
    rows, rhs = [], []
    for a, b in zip(x[:-1], x[1:]):
        xq = 0.5 * (b - a) * gx + 0.5 * (a + b)
        sw = np.sqrt(0.5 * (b - a) * gw)
        basis = np.stack([_pl_eval_1d(xc, np.eye(len(xc))[k], xq) for k in range(len(xc))], 1)
        rows.append(sw[:, None] * basis); rhs.append(sw * _pl_eval_1d(x, w, xq))
    zz = np.linalg.lstsq(np.concatenate(rows), np.concatenate(rhs), rcond=None)[0]
    np.testing.assert_allclose(z, zz, atol=1e-12)


# ------------------------------------------------------ brute force -------

def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


@pytest.mark.parametrize("dims,nonuni", [((9, 9), False), ((8, 6), True), ((5, 6, 7), True),
                                         ((9, 5, 9), False), ((4, 4, 4), True),
                                         ((5, 4, 5, 6), True), ((5, 5, 5, 5), False)])
def test_dense_kronecker_projection(dims, nonuni):
    """Q_{l-1} w equals the dense Galerkin projection with the full
    tensor-product matrices: (P^T M P)^{-1} P^T M w (numpy.linalg.solve)."""
    rng = _rng(5)
    coords = None
    if nonuni:
        coords = []
        for n in dims:
            x = np.cumsum(rng.uniform(0.2, 2.0, n)); coords.append(x)
    H = O.Hierarchy(dims, coords)
    w = rng.standard_normal(dims)
    ops = H.ops(H.L)
    M = _kron_all([o.Mf.toarray() for o in ops])
    P = _kron_all([o.P.toarray() for o in ops])
    z_dense = np.linalg.solve(P.T @ M @ P, P.T @ M @ w.ravel())
    z = O.project(w, H, H.L)
    np.testing.assert_allclose(z.ravel(), z_dense, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mass_matrix_integrates_exactly(seed):
    """On any grid the P1 mass matrix gives the exact L2 inner products of
    the functions the space holds: with 1 and x sampled at the nodes of
    [a, b], 1'M1 = b - a, 1'Mx = (b^2 - a^2)/2 and x'Mx = (b^3 - a^3)/3."""
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.uniform(0.1, 2.0, 9 + seed)) - 3.0
    a, b = x[0], x[-1]
    M = O.mass_matrix(x).toarray()
    one = np.ones_like(x)
    assert one @ M @ one == pytest.approx(b - a, rel=1e-13)
    assert one @ M @ x == pytest.approx((b * b - a * a) / 2, rel=1e-12, abs=1e-12)
    assert x @ M @ x == pytest.approx((b ** 3 - a ** 3) / 3, rel=1e-12)


def test_mass_matrix_three_nodes_by_hand():
    """x = (0, 1, 3): elements of length 1 and 2, each contributing
    h/3 on its diagonal and h/6 off it."""
    M = O.mass_matrix(np.array([0.0, 1.0, 3.0])).toarray()
    exp = np.array([[1 / 3, 1 / 6, 0.0], [1 / 6, 1.0, 1 / 3], [0.0, 1 / 3, 2 / 3]])
    np.testing.assert_allclose(M, exp, rtol=1e-15, atol=1e-16)


def test_galerkin_coarse_mass():
    """M_c assembled on the coarse coordinates equals P^T M_f P (nested P1
    spaces)."""
    rng = _rng(6)
    for n in (5, 6, 9, 12):
        x = np.cumsum(rng.uniform(0.1, 1.0, n))
        keep = O.coarse_indices(n)
        P = O.prolongation(x, keep)
        G = (P.T @ O.mass_matrix(x) @ P).toarray()
        np.testing.assert_allclose(O.mass_matrix(x[keep]).toarray(), G, atol=1e-14)


# -------------------------------------------------------- invariants -----

SHAPES = [(9,), (10,), (33,), (17, 17), (12, 9), (9, 9, 9), (10, 7, 12), (17, 9, 6)]


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("nonuni", [False, True])
def test_identity(dims, nonuni):
    """Recomposition inverts decomposition (Section 2) to 1e-12."""
    rng = _rng(7)
    coords = [F.geometric_coords(n, 1.03 + 0.02 * d) for d, n in enumerate(dims)] if nonuni else None
    H = O.Hierarchy(dims, coords)
    u = rng.standard_normal(dims)
    for stop in sorted({0, H.L // 2, H.L}):
        umc = O.decompose(u, H, stop)
        r = O.recompose(umc, H, stop)
        assert np.abs(r - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("dims", SHAPES)
def test_multilinear_input_zero_coefficients(dims):
    """Interpolation reproduces coarse-representable functions (Section 2),
    so multilinear input has zero coefficients at every level and the coarse
    block equals the input restricted to N_{l~}."""
    coords = [F.geometric_coords(n, 1.05) for n in dims]
    H = O.Hierarchy(dims, coords)
    u = F.multilinear_field(dims, coords)
    for stop in (0, max(0, H.L - 1)):
        umc = O.decompose(u, H, stop)
        lev = O.node_levels(H, stop)
        assert np.abs(umc[lev > stop]).max(initial=0) < 1e-13
        np.testing.assert_allclose(umc[np.ix_(*H.index[stop])], u[np.ix_(*H.index[stop])],
                                   atol=1e-13)


def test_piecewise_multilinear_on_coarse_level():
    """A function that is piecewise multilinear on N_k (built with scipy's
    linear grid interpolator) has zero coefficients at every level above k."""
    dims = (17, 12, 9)
    coords = [F.geometric_coords(n, 1.04) for n in dims]
    H = O.Hierarchy(dims, coords)
    k = H.L - 2
    ck = _rng(8).standard_normal(H.levels[k])
    fine = np.stack(np.meshgrid(*coords, indexing="ij"), -1)
    u = RegularGridInterpolator(H.coords[k], ck)(fine.reshape(-1, 3)).reshape(dims)
    umc = O.decompose(u, H, 0)
    lev = O.node_levels(H)
    assert np.abs(umc[lev > k]).max() < 1e-12
    assert np.abs(umc[lev == k]).max() > 1e-3


def test_paper_correction_identity():
    """Section 2 step 4: the projection of the multilevel component equals
    Q_{l-1}u - Pi_{l-1}Q_l u, i.e. Q_{l-1}u = u|_{N_{l-1}} + Q_{l-1}(mc)."""
    dims = (13, 10, 9)
    coords = [F.geometric_coords(n, 1.03) for n in dims]
    H = O.Hierarchy(dims, coords)
    u = _rng(9).standard_normal(dims)
    l = H.L
    keep = [o.keep for o in H.ops(l)]
    mc = u - O.interpolate(u[np.ix_(*keep)], H, l)
    lhs = O.project(u, H, l)
    rhs = u[np.ix_(*keep)] + O.project(mc, H, l)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(u).max()


def test_scale_shift_invariance():
    dims = (9, 10, 7)
    coords = [F.geometric_coords(n, 1.03) for n in dims]
    u = _rng(10).standard_normal(dims)
    a = O.decompose(u, O.Hierarchy(dims, coords))
    b = O.decompose(u, O.Hierarchy(dims, [17.0 * x - 3.0 for x in coords]))
    np.testing.assert_allclose(a, b, atol=1e-12)


# ---------------------------------------------------------- tolerances ----

def _exact_A(n):
    """A = M_c^{-1} P^T M_f for a uniform 1D grid, in exact rationals:
    mass matrices from the hat-function integrals h/3, h/6, Gauss-Jordan
    elimination in Fractions."""
    h = Fraction(1)
    Mf = [[Fraction(0)] * n for _ in range(n)]
    for j in range(n - 1):
        Mf[j][j] += h / 3; Mf[j + 1][j + 1] += h / 3
        Mf[j][j + 1] += h / 6; Mf[j + 1][j] += h / 6
    keep = list(range(0, n, 2)) + ([n - 1] if n % 2 == 0 else [])
    nc = len(keep)
    P = [[Fraction(0)] * nc for _ in range(n)]
    for k, j in enumerate(keep):
        P[j][k] = Fraction(1)
    for k in range(nc - 1):
        a, b = keep[k], keep[k + 1]
        for j in range(a + 1, b):
            P[j][k] = Fraction(b - j, b - a); P[j][k + 1] = Fraction(j - a, b - a)
    R = [[sum(P[i][k] * Mf[i][j] for i in range(n)) for j in range(n)] for k in range(nc)]
    Mc = [[sum(P[i][k] * sum(Mf[i][j] * P[j][m] for j in range(n)) for i in range(n))
           for m in range(nc)] for k in range(nc)]
    aug = [Mc[k][:] + R[k][:] for k in range(nc)]
    for c in range(nc):
        piv = aug[c][c]
        aug[c] = [v / piv for v in aug[c]]
        for r in range(nc):
            if r != c and aug[r][c] != 0:
                f = aug[r][c]
                aug[r] = [vr - f * vc for vr, vc in zip(aug[r], aug[c])]
    return [row[nc:] for row in aug], keep


@pytest.mark.parametrize("n,expected", [(5, Fraction(7, 4)), (9, Fraction(13, 7))])
def test_linf_constant_1d_exact(n, expected):
    """In 1D the constant is 1 + max_k (sum_j |A_kj| - sum_{j coarse} |A_kj|)
    (derivation in linf_constant); exact rational arithmetic for n = 5, 9."""
    A, keep = _exact_A(n)
    val = 1 + max(sum(abs(v) for v in row) - sum(abs(row[j]) for j in keep) for row in A)
    assert val == expected
    assert O.linf_constant(O.Hierarchy((n,))) == pytest.approx(float(expected), rel=1e-14)


def test_linf_constant_uniform_limit():
    """Large uniform grids: |A|_inf -> 1 + sqrt(3)/2 per axis (the rows of
    M_c^{-1} decay with ratio 2 - sqrt(3)), so C -> (1 + sqrt(3)/2)^d."""
    lim = 1 + np.sqrt(3) / 2
    for d in (1, 2, 3, 4):
        C = O.linf_constant(O.Hierarchy((129,) * d))
        assert C == pytest.approx(lim ** d, rel=1e-9)


def test_linf_constant_is_an_upper_bound_1d():
    """Worst case of one level: coefficient errors of +-1 with the signs of
    the row of K (coefficients -> correction) that attains its max row sum
    give a recomposition error of exactly that row sum at the coarse node;
    C must not be smaller than 1 + that, nor than the largest error."""
    n = 17
    H = O.Hierarchy((n,))
    l = H.L
    A = O.projection_matrix(H.ops(l)[0])
    keep = H.ops(l)[0].keep
    coef = np.setdiff1d(np.arange(n), keep)
    K = A[:, coef]
    k = np.argmax(np.abs(K).sum(1))
    e = np.zeros(n); e[coef] = np.sign(K[k])
    umc = np.zeros(n)
    umc[np.ix_(*H.index[l])] = e
    err = O.recompose(umc, H, l - 1)
    pos = H.index[l - 1][0][k]
    assert abs(err[pos]) == pytest.approx(np.abs(K[k]).sum(), rel=1e-12)
    C = O.linf_constant(H, l - 1)
    assert C >= 1 + np.abs(K[k]).sum() - 1e-12
    assert C >= np.abs(err).max()


@pytest.mark.parametrize("dims,nonuni", [((9, 7), False), ((5, 6, 5), True), ((5, 5, 4, 5), False),
                                         ((5, 4, 5, 5), True)])
def test_linf_constant_bounds_the_dense_operator(dims, nonuni):
    """In 2-4D the telescoping sum is an upper bound, not the exact norm:
    C_Linf must be at least 1 + the largest absolute row sum of the dense
    operator K (the Kronecker product of the axes' projections restricted to
    the coefficient columns) that maps the finest level's coefficients to
    the correction of the coarse values."""
    coords = [F.geometric_coords(n, 1.1) for n in dims] if nonuni else None
    H = O.Hierarchy(dims, coords)
    l = H.L
    ops = H.ops(l)
    A = O.projection_matrix(ops[0])
    for op in ops[1:]:
        A = np.kron(A, O.projection_matrix(op))
    coarse = np.zeros(dims, dtype=bool)
    coarse[np.ix_(*[op.keep for op in ops])] = True
    K = A[:, ~coarse.ravel()]
    true_norm = np.abs(K).sum(axis=1).max()
    C = O.linf_constant(H, l - 1)
    assert C >= 1 + true_norm - 1e-12
    # And the worst-case sign pattern of that row is reproduced by a
    # recomposition of coefficient errors alone.
    k = np.argmax(np.abs(K).sum(axis=1))
    e = np.zeros(int(np.prod(dims)))
    e[~coarse.ravel()] = np.sign(K[k])
    umc = np.zeros(dims)
    umc[np.ix_(*H.index[l])] = e.reshape(dims)
    err = O.recompose(umc, H, l - 1)
    pos = tuple(H.index[l - 1][d][i] for d, i in enumerate(np.unravel_index(k, H.levels[l - 1])))
    assert abs(err[pos]) == pytest.approx(true_norm, rel=1e-12)
    assert C >= np.abs(err).max()


@pytest.mark.parametrize("dims,stop", [((65,), 0), ((33, 17), 1), ((17, 17, 17), 0), ((20, 17, 9), 2)])
def test_tolerances_sum_and_ratio(dims, stop):
    """Eq. (LinfTau) / Algorithm 1: tau_{l+1} = kappa tau_l with
    kappa = sqrt(2^d), and sum_{l >= l~} tau_l = tau / C."""
    H = O.Hierarchy(dims)
    tau = 0.37
    C = O.linf_constant(H, stop)
    t = O.level_tolerances(H, stop, tau, C)
    kappa = np.sqrt(2.0 ** len(dims))
    np.testing.assert_allclose(t[stop + 1:] / t[stop:-1], kappa, rtol=1e-14)
    assert t[stop:].sum() == pytest.approx(tau / C, rel=1e-13)


def test_llround_matches_exact_rational_rounding():
    """Against rounding done in exact rational arithmetic (half away from
    zero) on random doubles of every magnitude up to 2^62, halves and their
    neighbours included."""
    from fractions import Fraction
    rng = np.random.default_rng(11)
    mags = 2.0 ** rng.uniform(-3, 62, 4000)
    y = np.concatenate([mags * rng.choice([-1.0, 1.0], mags.size),
                        np.arange(-40, 41) + 0.5,
                        np.nextafter(np.arange(-40, 41) + 0.5, np.inf),
                        np.nextafter(np.arange(-40, 41) + 0.5, -np.inf)])
    y = y[np.abs(y) < 2.0 ** 62]

    def exact(x):
        f = Fraction(float(x))
        r = int(abs(f) + Fraction(1, 2))  # floor(|x| + 1/2): int() truncates a positive value
        return r if f >= 0 else -r

    assert O.llround(y).tolist() == [exact(x) for x in y]


def test_llround_ties_and_edges():
    y = np.array([0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 0.49999999999999994,
                  -0.49999999999999994, 4503599627370495.5, 1e17, -3.0, 0.0])
    exp = np.array([1, -1, 2, -2, 3, -3, 0, 0, 4503599627370496, 10 ** 17, -3, 0])
    assert O.llround(y).tolist() == exp.tolist()


@pytest.mark.parametrize("dims,stop,nonuni", [((65,), 0, False), ((33, 33), 0, True),
                                               ((17, 19, 21), 0, False), ((17, 19, 21), 2, True)])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_linf_guarantee(dims, stop, nonuni, rel):
    """Eq. (LInfNormEstimator) with the level tolerances: quantize,
    dequantize and recompose; the max error stays within tau, and each
    coefficient is within its level tolerance."""
    coords = [F.geometric_coords(n, 1.03) for n in dims] if nonuni else None
    H = O.Hierarchy(dims, coords)
    u = F.grf_field(dims, seed=11, dtype=np.float64)
    tau = rel * O.value_range(u)
    taus = O.level_tolerances(H, stop, tau)
    umc = O.decompose(u, H, stop)
    k = O.quantize(umc, H, stop, taus)
    deq = O.dequantize(k, H, stop, taus)
    lev = O.node_levels(H, stop)
    assert np.all(np.abs(deq - umc) <= taus[lev] * (1 + 1e-12))
    rec = O.recompose(deq, H, stop)
    assert np.abs(rec - u).max() <= tau


def test_worst_case_quantization_errors_within_bound():
    """Adversarial coefficient errors: every coefficient off by +-tau_l with
    random signs (the extreme of each bin), many trials; still within tau."""
    dims = (17, 17)
    H = O.Hierarchy(dims)
    tau = 1.0
    taus = O.level_tolerances(H, 0, tau)
    lev = O.node_levels(H)
    rng = _rng(12)
    worst = 0.0
    for _ in range(50):
        e = taus[lev] * rng.choice([-1.0, 1.0], size=dims)
        worst = max(worst, np.abs(O.recompose(e, H, 0)).max())
    assert worst <= tau


# ------------------------------------------------ quantizer round trips ---

def test_value_range_and_quantizer_hand_values():
    """value_range, quantize and dequantize on hand-built values: bins of
    width 2 tau around zero, labels and centres worked out by hand."""
    u = np.array([-1.5, 0.25, 3.0, 2.0, -0.75])
    assert O.value_range(u) == 4.5
    assert O.value_range(np.float32([7.0, 7.0, 7.0])) == 0.0
    H = O.Hierarchy((5,))
    taus = np.full(H.L + 1, 0.25)       # every bin 0.5 wide
    x = np.array([0.24, -0.25, 0.75, -1.26, 100.0])
    # 0.48 -> 0; -0.5 -> -1 (tie away from zero); 1.5 -> 2 (tie); -2.52 -> -3; 200 -> 200
    k = O.quantize(x, H, 0, taus)
    assert k.tolist() == [0, -1, 2, -3, 200]
    back = O.dequantize(k, H, 0, taus)
    assert back.tolist() == [0.0, -0.5, 1.0, -1.5, 100.0]
    assert np.abs(back - x).max() <= 0.25


def test_dequantize_rounds_the_fp64_product_to_fp32():
    """Centres in FP32 are the FP64 products k q rounded once to FP32 (the
    value the label stands for), checked on products that need rounding."""
    H = O.Hierarchy((5,))
    q = 0.1  # tau = 0.05
    taus = np.full(H.L + 1, q / 2)
    k = np.array([1, 3, 7, -(2 ** 30) + 1, 123456789], dtype=np.int64)
    got = O.dequantize(k, H, 0, taus, dtype=np.float32)
    exp = np.array([np.float32(float(v) * 0.1) for v in k])
    assert np.array_equal(got, exp)


# ------------------------------------------- adaptive stopping level ---

def _pe_cases():
    cases = []
    with open(os.path.join(GOLDEN, "prediction_errors.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            dims_s, field_s, l_s, tau_s, el_s, ei_s = [p.strip() for p in line.split("|")]
            cases.append((tuple(int(v) for v in dims_s.split("x")), field_s, int(l_s),
                          float(tau_s), float(el_s), float(ei_s)))
    return cases


def _pe_field(dims, spec):
    if spec.startswith("spike"):
        v = np.zeros(dims)
        v[tuple(int(t) for t in spec.split()[1].split(","))] = 1.0
        return v
    assert spec == "xsq"
    i = np.arange(dims[0], dtype=np.float64)
    return np.broadcast_to((i * i)[:, None, None], dims).copy()


@pytest.mark.parametrize("case", _pe_cases())
def test_prediction_errors_hand_sums(case):
    dims, spec, l, tau0, e_lor, e_int = case
    H = O.Hierarchy(dims)
    got = O.prediction_errors(_pe_field(dims, spec), H, l, tau0)
    assert got[0] == pytest.approx(e_lor, rel=1e-12)
    assert got[1] == pytest.approx(e_int, rel=1e-12)


def test_sampled_blocks_one_in_four():
    # 17 nodes: cells [0,2], [2,4], .. [14,16]; cells 0 and 4 are sampled.
    # 10 nodes (even): coarse nodes 0,2,4,6,8,9; cells 0 and 4, the latter
    # the 2-node end cell [8,9].
    H = O.Hierarchy((17, 10, 5))
    b = O.sampled_blocks(H, H.L)
    assert b[0] == [(0, 2), (8, 10)]
    assert b[1] == [(0, 2), (8, 9)]
    assert b[2] == [(0, 2)]


def test_lorenzo_exact_where_mixed_difference_vanishes():
    # The 3D Lorenzo prediction error is the mixed third difference of u, so
    # it vanishes at interior nodes for any sum of functions each missing one
    # axis; there the estimate reduces to the penalties.  A product x*y*z
    # has mixed difference 1 and misses by exactly 1 everywhere inside.
    rng = _rng(5)
    dims = (9, 9, 9)
    f, g, h = rng.standard_normal((3, 9, 9))
    i, j, k = np.meshgrid(*[np.arange(9)] * 3, indexing="ij")
    u = f[i, j] + g[j, k] + h[i, k]
    xyz = (i * j * k).astype(np.float64)
    for x in range(1, 9):
        for y in range(1, 9):
            for z in range(1, 9):
                assert abs(O._lorenzo(u, (x, y, z)) - u[x, y, z]) < 1e-12
                assert abs(O._lorenzo(xyz, (x, y, z)) - xyz[x, y, z]) == pytest.approx(1.0)


def test_interp_estimate_of_multilinear_field_is_penalties_only():
    # Multilinear interpolation reproduces a multilinear field, so E_interp
    # is the penalty sum: per full block 12 edge, 6 plane, 1 cube nodes.
    dims = (17, 9, 13)
    coords = [F.geometric_coords(n, 1.05) for n in dims]
    H = O.Hierarchy(dims, coords)
    X, Y, Z = np.meshgrid(*coords, indexing="ij")
    u = 1.0 + 2.0 * X - Y + 0.5 * Z + 3.0 * X * Y - X * Y * Z
    tau0 = 0.3
    nblocks = np.prod([len(b) for b in O.sampled_blocks(H, H.L)])
    _, e_int = O.prediction_errors(u, H, H.L, tau0)
    assert e_int == pytest.approx(nblocks * (12 * 0.369 + 6 * 0.259 + 0.182) * tau0, rel=1e-10)


def test_adaptive_stop_level_decisions():
    H = O.Hierarchy((9, 9, 9))
    u = _pe_field((9, 9, 9), "xsq")
    # Small tau: Lorenzo (1 + 23.18 tau0) beats interpolation (9 + 6.16 tau0)
    # on the finest level, which becomes the stopping level.
    stop, sums = O.adaptive_stop_level(u, H, 1e-3)
    assert stop == H.L and list(sums) == [H.L]
    # Large tau: the Lorenzo penalty dominates; the finest level is decomposed.
    stop, sums = O.adaptive_stop_level(u, H, 1e3)
    assert stop < H.L and sums[H.L][0] > sums[H.L][1]
    # A 2D grid has no penalty factors in the paper.
    with pytest.raises(ValueError):
        O.prediction_errors(np.zeros((9, 9)), O.Hierarchy((9, 9)), 2, 1.0)


# --------------------------------- progressive recomposition, iso area ---

@pytest.mark.parametrize("dims,kind", [((17, 9, 12), "u"), ((10, 17, 9), "g")])
def test_recompose_partial_is_the_projection_chain(dims, kind):
    # Q_k u directly: the L2 projection applied level by level from the
    # finest grid (no decomposition involved).
    coords = None if kind == "u" else [F.geometric_coords(n, 1.04) for n in dims]
    H = O.Hierarchy(dims, coords)
    u = _rng(11).standard_normal(dims)
    for stop in (0, 1):
        umc = O.decompose(u, H, stop)
        v = u.copy()
        for k in range(H.L, stop - 1, -1):
            got = O.recompose_partial(umc, H, stop, k)
            np.testing.assert_allclose(got, v, atol=1e-12 * np.abs(u).max())
            if k > stop:
                v = O.project(v, H, k)


def test_iso_area_planes_exact():
    # Marching tetrahedra reproduce planar iso-surfaces exactly.
    n = (8, 6, 5)
    i, j, k = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij")
    assert O.iso_area(i, None, 3.5) == pytest.approx(5.0 * 4.0, rel=1e-13)
    n = (8, 8, 5)
    i, j, k = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in n], indexing="ij")
    # i + j = 4.3 cuts the (i, j) square along a segment of length 4.3 sqrt(2).
    assert O.iso_area(i + j, None, 4.3) == pytest.approx(4.3 * np.sqrt(2.0) * 4.0, rel=1e-13)
    # Nonuniform coordinates: the plane x = 0.37 spans the (y, z) extent.
    dims = (9, 7, 6)
    coords = [F.geometric_coords(n, 1.1) for n in dims]
    X, Y, Z = np.meshgrid(*coords, indexing="ij")
    ext = (coords[1][-1] - coords[1][0]) * (coords[2][-1] - coords[2][0])
    assert O.iso_area(X, coords, 0.37) == pytest.approx(ext, rel=1e-12)


def test_iso_area_sphere_converges():
    # r^2 = R^2 on grids of growing resolution approaches 4 pi R^2.
    errs = []
    for n, R in ((17, 6.0), (33, 12.0)):
        c = (n - 1) / 2
        i, j, k = np.meshgrid(*[np.arange(n, dtype=np.float64)] * 3, indexing="ij")
        r2 = (i - c) ** 2 + (j - c) ** 2 + (k - c) ** 2
        errs.append(abs(O.iso_area(r2, None, R * R) / (4 * np.pi * R * R) - 1))
    assert errs[0] < 0.02 and errs[1] < errs[0]


# ------------------------------------------------ lossless stage, PSNR ---

def _packed_cases():
    out = []
    with open(os.path.join(GOLDEN, "packed_labels.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            labels_s, hex_s = [p.strip() for p in line.split("|")]
            out.append(([int(v) for v in labels_s.split(",")], bytes.fromhex(hex_s.replace(" ", ""))))
    return out


@pytest.mark.parametrize("case", _packed_cases())
def test_pack_labels_hand_streams(case):
    labels, stream = case
    assert O.pack_labels(labels) == stream
    assert list(O.unpack_labels(stream)) == labels


def test_pack_labels_round_trip_and_size():
    rng = _rng(9)
    for n in (0, 1, 1023, 1024, 1025, 5000):
        x = rng.integers(-40, 40, n)
        if n > 10:
            x[3] = 2 ** 62
            x[n - 1] = -2 ** 63
            x[n // 2] = 2 ** 63 - 1
        buf = O.pack_labels(x)
        assert np.array_equal(O.unpack_labels(buf), x)
        # Size: header, widths padded to 8 bytes, then ceil(n_c w / 64) words.
        nch = (n + 1023) // 1024
        size = 8 + nch + (-(8 + nch)) % 8
        for c in range(nch):
            z = [(2 * int(v)) if v >= 0 else (-2 * int(v) - 1) for v in x[c * 1024:(c + 1) * 1024]]
            w = max(z).bit_length()
            size += 8 * ((len(z) * w + 63) // 64)
        assert len(buf) == size


def test_psnr_closed_form():
    u = np.array([0.0, 1.0])
    v = np.array([0.0, 1.1])
    # range 1, mean squared error 0.005
    assert O.psnr(u, v) == pytest.approx(-10 * np.log10(0.005), rel=1e-14)


def test_psnr_uses_the_range_of_the_original():
    """The range term is max u - min u (the reading of the garbled printed
    formula): a reconstruction whose minimum differs from the original's
    (here 0.1 against 0) must not change it, and a uniform offset e of a
    field of range R gives 20 log10(R / |e|)."""
    u = np.array([0.0, 1.0])
    v = np.array([0.1, 1.0])
    assert O.psnr(u, v) == pytest.approx(-10 * np.log10(0.005), rel=1e-14)
    w = np.random.default_rng(3).uniform(-2.0, 5.0, (7, 5, 3))
    R = float(w.max() - w.min())
    assert O.psnr(w, w + 0.01) == pytest.approx(20 * np.log10(R / 0.01), rel=1e-12)
    assert O.psnr(w, w - 0.01) == pytest.approx(20 * np.log10(R / 0.01), rel=1e-12)


# --------------------------------------- L-inf-optimal and L2 bin widths ---

def test_l2_tolerances_uniform_closed_form():
    # 5^3 with index coordinates: h_1 = 1, h_0 = 2, #N_L = 125.
    H = O.Hierarchy((5, 5, 5))
    t = O.level_tolerances_mode(H, 0, 1.0, "l2")
    assert t[1] == pytest.approx(1.0 / np.sqrt(125.0), rel=1e-14)
    assert t[0] == pytest.approx(1.0 / np.sqrt(8.0 * 125.0), rel=1e-14)
    # Geometric growth kappa = 2^(d/2) on dyadic grids (Section 4.1).
    H = O.Hierarchy((33, 17, 9))
    t = O.level_tolerances_mode(H, 1, 2.0, "l2")
    np.testing.assert_allclose(t[2:] / t[1:-1], np.sqrt(8.0), rtol=1e-13)


def _worst_errors(H, stop, taus, seed):
    # Coefficient errors of magnitude tau_l with random signs at every node.
    rng = _rng(seed)
    lev = O.node_levels(H, stop)
    return np.asarray(taus)[lev] * rng.choice([-1.0, 1.0], size=lev.shape)


@pytest.mark.parametrize("dims,kind,stop", [((17, 17, 9), "u", 0), ((12, 10, 9), "g", 1),
                                            ((33, 17), "g", 0)])
def test_l2_bound_holds_for_worst_errors(dims, kind, stop):
    coords = None if kind == "u" else [F.geometric_coords(n, 1.08) for n in dims]
    H = O.Hierarchy(dims, coords)
    tau = 0.3
    taus = O.level_tolerances_mode(H, stop, tau, "l2")
    for seed in range(3):
        err = O.recompose(_worst_errors(H, stop, taus, seed), H, stop)
        assert O.l2_error(err, H) <= tau * (1 + 1e-12)


@pytest.mark.parametrize("n,h", [(5, 1.0), (9, 0.25), (17, 3.0)])
def test_l2_error_unit_hat_closed_form(n, h):
    # One unit nodal value at an interior node of a uniform 1D grid of
    # spacing h is a hat function: its squared L2 norm is 2h/3.  The norm
    # (not its square) is returned, and h enters to the power 1/2.
    H = O.Hierarchy((n,), [h * np.arange(n, dtype=np.float64)])
    e = np.zeros(n)
    e[n // 2] = 1.0
    assert O.l2_error(e, H) == pytest.approx(math.sqrt(2.0 * h / 3.0), rel=1e-14)
    # An end node carries half a hat: h/3.
    e = np.zeros(n)
    e[0] = 1.0
    assert O.l2_error(e, H) == pytest.approx(math.sqrt(h / 3.0), rel=1e-14)


@pytest.mark.parametrize("dims", [(7,), (9, 5), (5, 6, 7), (4, 5, 3, 6)])
def test_l2_error_constant_on_unit_box(dims):
    # A constant c on [0,1]^d (any node spacing) has L2 norm |c|: every axis
    # of the tensor mass product must contribute its full length 1.
    rng = _rng(11)
    coords = [np.concatenate([[0.0], np.sort(rng.uniform(0, 1, n - 2)), [1.0]]) for n in dims]
    H = O.Hierarchy(dims, coords)
    c = -2.75
    assert O.l2_error(np.full(dims, c), H) == pytest.approx(abs(c), rel=1e-13)
    # On a box of side lengths a_d the norm is |c| sqrt(prod a_d).
    a = [1.0 + 0.5 * d for d in range(len(dims))]
    H = O.Hierarchy(dims, [a[d] * coords[d] for d in range(len(dims))])
    assert O.l2_error(np.full(dims, c), H) == pytest.approx(abs(c) * math.sqrt(np.prod(a)),
                                                             rel=1e-13)


def test_l2_error_multilinear_product_closed_form():
    # A product of linear factors is reproduced exactly by the P1 function,
    # so its norm is the product of the 1D integrals (closed form) on a
    # nonuniform 3D grid: int_0^1 (1 + 2x)^2 = 13/3, int_0^1 y^2 = 1/3,
    # int_0^1 (2 - z)^2 = 7/3.
    dims = (6, 7, 5)
    coords = [np.concatenate([[0.0], np.sort(_rng(s).uniform(0, 1, n - 2)), [1.0]])
              for s, n in zip((3, 4, 5), dims)]
    H = O.Hierarchy(dims, coords)
    X, Y, Z = np.meshgrid(*coords, indexing="ij")
    e = (1 + 2 * X) * Y * (2 - Z)
    exact = math.sqrt(13.0 / 3.0 * 1.0 / 3.0 * 7.0 / 3.0)
    assert O.l2_error(e, H) == pytest.approx(exact, rel=1e-13)


def test_l2_error_piecewise_linear_by_quadrature():
    # An arbitrary P1 function on nonuniform 1D and 2D grids, integrated
    # cell by cell with 3-point Gauss-Legendre quadrature (exact for the
    # squared piecewise-(bi)linear integrand) by an evaluator that does not
    # use the mass matrix.
    gx, gw = np.polynomial.legendre.leggauss(3)
    rng = _rng(21)
    x = np.cumsum(rng.uniform(0.2, 1.5, 8))
    y = np.cumsum(rng.uniform(0.3, 1.1, 6))
    e2 = rng.standard_normal((8, 6))
    e1 = e2[:, 2].copy()

    def cell_pts(a, b):
        return 0.5 * (b - a) * gx + 0.5 * (a + b), 0.5 * (b - a) * gw

    s1 = 0.0
    for i in range(len(x) - 1):
        p, w = cell_pts(x[i], x[i + 1])
        t = (p - x[i]) / (x[i + 1] - x[i])
        s1 += float(np.sum(w * ((1 - t) * e1[i] + t * e1[i + 1]) ** 2))
    assert O.l2_error(e1, O.Hierarchy((8,), [x])) == pytest.approx(math.sqrt(s1), rel=1e-13)

    s2 = 0.0
    for i in range(len(x) - 1):
        px, wx = cell_pts(x[i], x[i + 1])
        tx = (px - x[i]) / (x[i + 1] - x[i])
        for j in range(len(y) - 1):
            py, wy = cell_pts(y[j], y[j + 1])
            ty = (py - y[j]) / (y[j + 1] - y[j])
            TX, TY = np.meshgrid(tx, ty, indexing="ij")
            f = ((1 - TX) * (1 - TY) * e2[i, j] + TX * (1 - TY) * e2[i + 1, j]
                 + (1 - TX) * TY * e2[i, j + 1] + TX * TY * e2[i + 1, j + 1])
            s2 += float(np.sum(np.outer(wx, wy) * f ** 2))
    assert O.l2_error(e2, O.Hierarchy((8, 6), [x, y])) == pytest.approx(math.sqrt(s2), rel=1e-13)


@pytest.mark.parametrize("dims,kind,stop", [((17, 17, 9), "u", 0), ((12, 10, 9), "g", 1)])
def test_linf_optimal_widths(dims, kind, stop):
    coords = None if kind == "u" else [F.geometric_coords(n, 1.08) for n in dims]
    H = O.Hierarchy(dims, coords)
    tau = 0.3
    taus = O.level_tolerances_mode(H, stop, tau, "linf_optimal")
    # Proportional to the level's node count, summing to tau / C_Linf.
    counts = [np.prod(H.levels[stop])] + [np.prod(H.levels[l]) - np.prod(H.levels[l - 1])
                                          for l in range(stop + 1, H.L + 1)]
    np.testing.assert_allclose(taus[stop:] / np.asarray(counts, dtype=float),
                               taus[stop] / counts[0], rtol=1e-13)
    assert taus[stop:].sum() == pytest.approx(tau / O.linf_constant(H, stop), rel=1e-13)
    for seed in range(3):
        err = O.recompose(_worst_errors(H, stop, taus, seed), H, stop)
        assert np.abs(err).max() <= tau * (1 + 1e-12)


# -------------------------------------------- coarse-part Lorenzo coder ---

def test_lorenzo_residuals_by_hand():
    # On a 3^3 coarse block: a constant leaves one residual, at the origin
    # (no lower neighbours); q = i (the axis-0 index) leaves 1 on the line
    # j = k = 0 for i >= 1 (every other node's mixed difference vanishes).
    H = O.Hierarchy((3, 3, 3))
    r = O.lorenzo_encode(np.full((3, 3, 3), 5, dtype=np.int64), H, 0)
    exp = np.zeros((3, 3, 3), dtype=np.int64)
    exp[0, 0, 0] = 5
    assert np.array_equal(r, exp)
    q = np.broadcast_to(np.arange(3)[:, None, None], (3, 3, 3)).astype(np.int64)
    exp = np.zeros((3, 3, 3), dtype=np.int64)
    exp[1, 0, 0] = exp[2, 0, 0] = 1
    assert np.array_equal(O.lorenzo_encode(q, H, 0), exp)


@pytest.mark.parametrize("dims,stop", [((17, 9, 12), 0), ((17, 9, 12), 2), ((33, 20), 1),
                                       ((100,), 3)])
def test_lorenzo_round_trip_and_scope(dims, stop):
    H = O.Hierarchy(dims)
    x = _rng(2).integers(-2 ** 62, 2 ** 62, dims)
    e = O.lorenzo_encode(x, H, stop)
    assert np.array_equal(O.lorenzo_decode(e, H, stop), x)
    # Only the coarse block changes.
    mask = np.zeros(dims, dtype=bool)
    mask[np.ix_(*H.index[stop])] = True
    assert np.array_equal(e[~mask], x[~mask])



# ----------------------------------------------------------- 4D grids ---

@pytest.mark.parametrize("dims", [(9, 5, 7, 6), (17, 9, 9, 5)])
def test_4d_multilinear_zero_coefficients_and_identity(dims):
    # The 4D hierarchy (QMCPACK's shape class, Section 6): multilinear input
    # has zero coefficients at every level; decompose-then-recompose is the
    # identity to 1e-12.
    coords = [F.geometric_coords(n, 1.05) for n in dims]
    H = O.Hierarchy(dims, coords)
    u = F.multilinear_field(dims, coords)
    umc = O.decompose(u, H, 0)
    lev = O.node_levels(H)
    assert np.abs(umc[lev > 0]).max() < 1e-12
    x = _rng(4).standard_normal(dims)
    r = O.recompose(O.decompose(x, H, 0), H, 0)
    assert np.abs(r - x).max() <= 1e-12 * np.abs(x).max()
    # kappa = sqrt(2^4) = 4 between consecutive level tolerances.
    t = O.level_tolerances(H, 0, 1.0)
    np.testing.assert_allclose(t[1:] / t[:-1], 4.0, rtol=1e-13)


# ---------------------------------------------------------------------------
# Entropy, cost model and the Huffman coder of the labels
# ---------------------------------------------------------------------------

def test_label_entropy_closed_forms():
    assert O.label_entropy([]) == 0.0
    assert O.label_entropy([7] * 10) == 0.0
    for k in (1, 3, 6):
        x = np.repeat(np.arange(-(2 ** (k - 1)), 2 ** (k - 1)), 5)
        assert O.label_entropy(x) == pytest.approx(k, abs=1e-12)
    p = 0.2
    x = [0] * 200 + [1] * 800
    assert O.label_entropy(x) == pytest.approx(-p * math.log2(p) - (1 - p) * math.log2(1 - p), abs=1e-12)


def test_cost_model_hand_count():
    # 1D, 5 nodes: N_0 has 3 nodes, N*_1 the other 2.  Full depth:
    # 3 log2(R / q_0) + 2 log2(R / q_1) with q_l = 2 tau_l.
    H = O.Hierarchy((5,))
    taus = [0.125, 0.25]
    assert O.cost_model(H, 0, taus, 8.0) == pytest.approx(3 * math.log2(32) + 2 * math.log2(16))
    # Stopping at level 1 counts the whole grid with tau_1.
    assert O.cost_model(H, 1, taus, 8.0) == pytest.approx(5 * math.log2(16))


def test_huffman_lengths_textbook_example():
    # The classic six-symbol example (counts 45, 13, 12, 16, 9, 5): the
    # optimal code lengths are 1, 3, 3, 3, 4, 4 (224 bits per 100 symbols).
    L = O.huffman_lengths([45, 13, 12, 16, 9, 5])
    assert L == [1, 3, 3, 3, 4, 4]


def _optimal_cost_brute(counts):
    """Least sum c_i L_i over length vectors meeting Kraft's equality (every
    full binary tree), by enumeration for a handful of symbols."""
    n = len(counts)
    best = None
    for Ls in itertools.product(range(1, n), repeat=n):
        if sum(2.0 ** -L for L in Ls) == 1.0:
            cost = sum(c * L for c, L in zip(counts, Ls))
            best = cost if best is None else min(best, cost)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_huffman_lengths_optimal_and_kraft(seed):
    rng = _rng(40 + seed)
    n = int(rng.integers(2, 6))
    counts = [int(v) for v in rng.integers(1, 50, n)]
    L = O.huffman_lengths(counts)
    assert sum(2.0 ** -l for l in L) == 1.0
    assert sum(c * l for c, l in zip(counts, L)) == _optimal_cost_brute(counts)
    # Average length within [H, H + 1) (the entropy bound of Section 4.1's
    # cost estimate).
    p = np.asarray(counts, dtype=np.float64) / sum(counts)
    Hs = float(-(p * np.log2(p)).sum())
    avg = sum(c * l for c, l in zip(counts, L)) / sum(counts)
    assert Hs - 1e-12 <= avg < Hs + 1.0


def test_huffman_length_limit():
    # Fibonacci counts make the unlimited Huffman tree a chain of depth
    # n - 1; with 40 symbols the limit (31 bits) must engage.
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    L = O.huffman_lengths(fib)
    assert max(L) <= 31
    assert sum(2.0 ** -l for l in L) == 1.0
    # Below the limit the chain is kept: 20 Fibonacci counts, depth 19.
    assert max(O.huffman_lengths(fib[:20])) == 19


def _huffman_cases():
    out = []
    with open(os.path.join(GOLDEN, "huffman_streams.txt")) as fh:
        for line in fh:
            line = line.rstrip("\n")
            if not line.strip() or line.startswith("#"):
                continue
            f = [p.strip() for p in line.split("|")]
            labels = [int(v) for v in f[0].split(",")]
            lengths = {int(a): int(b) for a, b in (t.split(":") for t in f[1].split(","))}
            chunks = [int(v) for v in f[2].split(",")]
            payload = bytes.fromhex(f[3].replace(" ", ""))
            out.append((labels, lengths, chunks, payload))
    return out


@pytest.mark.parametrize("case", _huffman_cases())
def test_huffman_hand_streams(case):
    labels, lengths, chunks, payload = case
    buf = O.huffman_encode(labels)
    K = O.HUFF_K
    assert int.from_bytes(buf[0:8], "little") == len(labels)
    assert int.from_bytes(buf[8:12], "little") == K == 32817
    assert int.from_bytes(buf[12:16], "little") == max(lengths.values())
    table = buf[16:16 + K]
    assert {s: table[s] for s in range(K) if table[s]} == lengths
    off = 16 + K
    assert buf[off:off + (-off) % 8] == bytes((-off) % 8)
    off += (-off) % 8
    got = [int.from_bytes(buf[off + 4 * c:off + 4 * c + 4], "little") for c in range(len(chunks))]
    assert got == chunks
    off += 4 * len(chunks)
    off += (-off) % 8
    assert buf[off:] == payload
    assert list(O.huffman_decode(buf)) == labels


def test_huffman_round_trip():
    rng = _rng(77)
    assert O.huffman_decode(O.huffman_encode([])).size == 0
    for n in (1, 1023, 1024, 1025, 3000):
        x = (rng.geometric(0.1, n) - 1) * rng.choice([-1, 1], n)
        if n > 10:
            x[2] = 2 ** 62
            x[n - 1] = -2 ** 63      # zigzag 2^64 - 1: bit length 64
            x[n // 2] = 2 ** 63 - 1
            x[5] = 16383             # zigzag 32766, the last direct symbols
            x[6] = -16384            # zigzag 32767
            x[7] = 16384             # zigzag 32768: bit length 16, 15 extra bits
        buf = O.huffman_encode(x)
        assert np.array_equal(O.huffman_decode(buf), x)
        # The payload is within one bit per label of the entropy of the
        # symbols plus the extra bits.
        z = [O._zigzag(int(v)) for v in x]
        parts = [O._huff_symbol(v) for v in z]
        sym = np.asarray([p[0] for p in parts])
        extra = sum(p[2] for p in parts)
        nchunks = (n + 1023) // 1024
        off = 16 + O.HUFF_K
        off += (-off) % 8 + 4 * nchunks
        off += (-off) % 8
        payload_bits = 8 * (len(buf) - off)
        assert payload_bits <= n * (O.label_entropy(sym) + 1) + extra + 64 * nchunks


@pytest.mark.parametrize("seed", range(4))
def test_huffman_cost_matches_heap_construction(seed):
    """Any Huffman construction gives the same total cost: the sum of the
    weights of the merged nodes.  A textbook heap-based merge (independent of
    the two-queue form used by the oracle) must give the cost of the
    oracle's lengths, on alphabets of hundreds of symbols."""
    import heapq
    rng = _rng(500 + seed)
    counts = [int(c) for c in rng.integers(1, 10 ** 6, int(rng.integers(50, 600)))]
    L = O.huffman_lengths(counts)
    heap = list(counts)
    heapq.heapify(heap)
    cost = 0
    while len(heap) > 1:
        a = heapq.heappop(heap)
        b = heapq.heappop(heap)
        cost += a + b
        heapq.heappush(heap, a + b)
    assert sum(c * l for c, l in zip(counts, L)) == cost
