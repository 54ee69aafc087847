"""GPU parity of the 4D grids (Section 2's hierarchy with d = 4) with the FP64
oracle: decomposition and recomposition element by element, the level-wise
quantizer bit-exact given the same coefficients and tolerances, and the
compressed round trip within the L-inf bound.

Tolerances as for 1-3D (tests/tolerances.py): FP64 within 1e-12 max|u|,
FP32 within 24 u (L + 1) max|u| with u = 2^-24 (four axes of operators with
max norm < 2 and a few dozen roundings per value and level)."""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F
from tolerances import TOL64, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2010_05872_gb300 import build as build_mod
    build_mod.build()
    B.lib()
    return torch


def _coords(dims, kind):
    if kind == "u":
        return None
    return [F.geometric_coords(n, 1.03 + 0.02 * d) for d, n in enumerate(dims)]


CASES = [((9, 5, 7, 6), "u", 0), ((9, 9, 9, 9), "u", 0), ((17, 9, 10, 9), "g", 0),
         ((17, 9, 10, 9), "g", 1), ((12, 17, 9, 33), "g", 0), ((17, 17, 17, 17), "u", 1),
         ((3, 3, 3, 3), "u", 0)]


@pytest.mark.parametrize("dims,kind,stop", CASES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_decompose_recompose_4d(cuda, dims, kind, stop, dtype):
    torch = cuda
    coords = _coords(dims, kind)
    H = O.Hierarchy(dims, coords)
    stop = min(stop, H.L)
    u = F.sinusoid_field(dims, seed=11).astype(dtype)
    exp = O.decompose(u.astype(np.float64), H, stop)
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    B.decompose_4d(x, coords, stop)
    scale = np.abs(u).max()
    tol = TOL64 if dtype == np.float64 else tol32(H.L)
    got = x.cpu().numpy().astype(np.float64)
    assert np.abs(got - exp).max() / scale <= tol
    # Recomposition of the oracle's coefficients, and the GPU round trip.
    y = torch.from_numpy(exp.astype(dtype)).cuda()
    B.recompose_4d(y, coords, stop)
    exp_r = O.recompose(exp.astype(dtype).astype(np.float64), H, stop)
    assert np.abs(y.cpu().numpy().astype(np.float64) - exp_r).max() / scale <= tol
    B.recompose_4d(x, coords, stop)
    assert np.abs(x.cpu().numpy().astype(np.float64) - u.astype(np.float64)).max() / scale <= tol


def test_multilinear_field_has_zero_coefficients_4d(cuda):
    torch = cuda
    dims = (17, 9, 10, 9)
    coords = _coords(dims, "g")
    H = O.Hierarchy(dims, coords)
    u = F.multilinear_field(dims, coords, seed=3)
    x = torch.from_numpy(u.copy()).cuda()
    B.decompose_4d(x, coords, 0)
    got = x.cpu().numpy()
    mask = np.ones(dims, dtype=bool)
    mask[np.ix_(*H.index[0])] = False
    assert np.abs(got[mask]).max() <= 1e-12 * np.abs(u).max()
    np.testing.assert_allclose(got[np.ix_(*H.index[0])], u[np.ix_(*H.index[0])], atol=1e-12)


@pytest.mark.parametrize("dims,kind,stop", [((17, 9, 10, 9), "g", 0), ((17, 17, 17, 17), "u", 1)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_quantize_4d_bit_exact_and_bound(cuda, dims, kind, stop, dtype):
    torch = cuda
    coords = _coords(dims, kind)
    H = O.Hierarchy(dims, coords)
    u = F.sinusoid_field(dims, seed=5).astype(dtype)
    tau = 1e-3 * O.value_range(u)
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    B.decompose_4d(x, coords, stop)
    labels, taus = B.quantize_4d(x, tau, coords, stop)
    np.testing.assert_allclose(taus, O.level_tolerances(H, stop, tau), rtol=1e-12)
    coeffs = x.cpu().numpy().astype(np.float64)
    exp = O.quantize(coeffs, H, stop, taus)
    assert np.array_equal(labels.cpu().numpy(), exp)
    deq = B.dequantize_4d(labels, tau, x.dtype, coords, stop)
    assert np.array_equal(deq.cpu().numpy(), O.dequantize(exp, H, stop, taus, dtype=dtype))
    B.recompose_4d(deq, coords, stop)
    err = np.abs(deq.cpu().numpy().astype(np.float64) - u.astype(np.float64)).max()
    eps = 1e-9 if dtype == np.float64 else tol32(H.L) * np.abs(u).max()
    assert err <= tau + eps


def test_errors_4d(cuda):
    torch = cuda
    x = torch.zeros((9, 9, 9, 9), device="cuda")
    with pytest.raises(B.MgardError) as e:
        B.decompose_4d(x, None, 3)
    assert e.value.code == -4
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.MgardError) as e:
        B.decompose_4d(x, None, 0, ws=ws)
    assert e.value.code == -5
    x[1, 2, 3, 4] = float("nan")
    with pytest.raises(B.MgardError) as e:
        B.quantize_4d(x, 0.1)
    assert e.value.code == -7
    # stop_level = L leaves the array as it is.
    y = torch.arange(81.0, device="cuda").reshape(3, 3, 3, 3)
    B.decompose_4d(y, None, 0)
    assert torch.equal(y, torch.arange(81.0, device="cuda").reshape(3, 3, 3, 3))
